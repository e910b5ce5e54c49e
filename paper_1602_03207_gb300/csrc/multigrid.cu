// Aggregation multigrid preconditioner built on the subdomain blocks.
//
// The paper partitions the mesh into subdomains (Sec. 3, Step 2).  Here the
// subdomains are (i) the smoothing blocks of the finest level (block-Jacobi
// with dense block inverses, kernel (c)) and (ii) the aggregates of the first
// coarsening: every subdomain becomes one coarse node with four unknowns
// (A_x, A_y, A_z, V).  The tentative prolongator carries the near-null
// vectors of the operator (a constant field per component): on the finest
// level its weights are 1/t (t the diagonal scaling) on free unknowns and 0
// on constrained ones, on coarser levels 1 on non-empty and 0 on empty coarse
// unknowns.  The coarse operator is the Galerkin product E = P^T A P (plus
// the identity on empty coarse unknowns); it is again a matrix of 4x4 complex
// blocks, so the same BSR SpMV and block kernels serve every level.  Coarse
// levels are aggregated greedily (a seed takes its not yet aggregated
// neighbours in increasing order, at most 8 nodes) and renumbered so that
// aggregates are contiguous; the coarsest level (<= 2048 unknowns) is
// inverted densely.  The cycle is a W-cycle with one block-Jacobi sweep
// before and after the coarse corrections.  On the levels above 16k nodes the
// residual after each coarse correction z += P e is updated as t -= (AP) e
// instead of recomputed (AP = A P, built next to the Galerkin product); the
// small levels recompute it with the warp-per-row SpMM.
//
// Setup runs once per matrix: patterns and aggregation on the host (integer
// work), Galerkin values on the device (one thread per coarse block sums its
// fine blocks in a fixed order).
#include <algorithm>
#include <numeric>
#include <deque>
#include <type_traits>

#include "common.cuh"

namespace {

constexpr int AGG_SIZE = 8;
constexpr int64_t WARP_ROW_MAX_NODES = 16384;  // levels up to this size use the warp-per-row SpMM
constexpr int64_t MAX_COARSE_DOFS = 2048;

// coarse block values: sum over the fine blocks mapped to each coarse block of
// w_i[p] A_ij[p][q] w_j[q]; identity on empty coarse unknowns of diagonal blocks
__global__ void k_galerkin(const int32_t* __restrict__ cptr, const int32_t* __restrict__ clist,
                           const int32_t* __restrict__ frow, const int32_t* __restrict__ fcol,
                           const double2* __restrict__ fval, const double* __restrict__ w, int64_t nnzc,
                           const int32_t* __restrict__ crow_of_slot, const int32_t* __restrict__ ccol,
                           const uint8_t* __restrict__ cempty, double2* __restrict__ cval) {
    const int64_t cs = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (cs >= nnzc) return;
    double re[16], im[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) re[e] = im[e] = 0.0;
    for (int32_t q = cptr[cs]; q < cptr[cs + 1]; ++q) {
        const int32_t s = clist[q];
        const int64_t i = frow[s], j = fcol[s];
        double wi[4], wj[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            wi[p] = w[4 * i + p];
            wj[p] = w[4 * j + p];
        }
        const double2* v = fval + 16 * (int64_t)s;
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const double f = wi[p] * wj[r];
                re[4 * p + r] += f * v[4 * p + r].x;
                im[4 * p + r] += f * v[4 * p + r].y;
            }
    }
    const int32_t I = crow_of_slot[cs], J = ccol[cs];
    double2* out = cval + 16 * cs;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            double2 v = make_double2(re[4 * p + r], im[4 * p + r]);
            if (I == J && p == r && cempty[4 * (int64_t)I + p]) v = make_double2(1.0, 0.0);
            out[4 * p + r] = v;
        }
}

// rc[r][4 I + p] = sum over the fine nodes i of coarse node I of w[4 i + p] t[r][4 i + p]
template <typename T>
__global__ void k_restrict(const C<T>* __restrict__ t, int64_t ldf, const int32_t* __restrict__ lo,
                           const int32_t* __restrict__ hi, const T* __restrict__ w, int64_t nc_nodes, int k,
                           const int* __restrict__ active, C<T>* __restrict__ rc, int64_t ldc) {
    const int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (d >= 4 * nc_nodes || (active && !active[r])) return;
    const int64_t I = d >> 2;
    const int p = (int)(d & 3);
    C<T> s = czero<T>();
    for (int32_t i = lo[I]; i < hi[I]; ++i) {
        const T wi = w[4 * (int64_t)i + p];
        const C<T> v = t[(int64_t)r * ldf + 4 * (int64_t)i + p];
        s.x += wi * v.x;
        s.y += wi * v.y;
    }
    rc[(int64_t)r * ldc + d] = s;
}

// z[r][4 i + p] += w[4 i + p] zc[r][4 agg(i) + p]
template <typename T>
__global__ void k_prolong(C<T>* __restrict__ z, int64_t ldf, const int32_t* __restrict__ node_agg,
                          const T* __restrict__ w, int64_t n_nodes, const C<T>* __restrict__ zc, int64_t ldc,
                          const int* __restrict__ active) {
    const int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (d >= 4 * n_nodes || (active && !active[r])) return;
    const T wi = w[d];
    if (wi == T(0)) return;
    const C<T> v = zc[(int64_t)r * ldc + 4 * (int64_t)node_agg[d >> 2] + (d & 3)];
    C<T>& o = z[(int64_t)r * ldf + d];
    o.x += wi * v.x;
    o.y += wi * v.y;
}

// Values of AP (A times the tentative prolongator, fine rows x coarse
// columns): block (i, J) sums A_ij diag(w_j) over the fine columns j of coarse
// node J, in ascending fine-block order.
__global__ void k_ap_values(const int32_t* __restrict__ src_ptr, const int32_t* __restrict__ src,
                            const int32_t* __restrict__ fcol, const double2* __restrict__ fval,
                            const double* __restrict__ w, int64_t nnz_ap, double2* __restrict__ out) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nnz_ap) return;
    double re[16], im[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) re[e] = im[e] = 0.0;
    for (int32_t q = src_ptr[b]; q < src_ptr[b + 1]; ++q) {
        const int32_t s = src[q];
        const int64_t j = fcol[s];
        const double2* v = fval + 16 * (int64_t)s;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const double wj = w[4 * j + c];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                re[4 * r + c] += v[4 * r + c].x * wj;
                im[4 * r + c] += v[4 * r + c].y * wj;
            }
        }
    }
#pragma unroll
    for (int e = 0; e < 16; ++e) out[16 * b + e] = make_double2(re[e], im[e]);
}

// t[r][4 i + p] -= sum over the blocks (i, J) of AP of AP_iJ[p][:] e[r][4 J + :].
// After a coarse correction z += P e, the new residual r - A z equals t - AP e:
// AP holds a third of A's blocks and e is a small coarse vector that stays in
// L2, so this costs a fraction of a full residual SpMM.  Tiles of KT
// right-hand sides are full; masked ones are computed and not stored.
template <typename T, int KT>
__global__ void __launch_bounds__(256) k_ap_update(const int32_t* __restrict__ ap_ptr,
                                                   const int32_t* __restrict__ ap_col,
                                                   const C<T>* __restrict__ ap_val, const C<T>* __restrict__ e,
                                                   int64_t lde, C<T>* __restrict__ t, int64_t ldt, int64_t n_rows,
                                                   const int* __restrict__ active, int ntile) {
    const int tile = (int)(blockIdx.x % ntile);
    const int64_t d = (int64_t)(blockIdx.x / ntile) * blockDim.x + threadIdx.x;
    if (d >= 4 * n_rows) return;
    const int row = (int)(d >> 2), p = (int)(d & 3);
    const int r0 = tile * KT;
    bool any = false;
#pragma unroll
    for (int q = 0; q < KT; ++q) any |= !active || active[r0 + q];
    if (!any) return;  // the whole tile has retired
    C<T> acc[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) acc[q] = czero<T>();
    const int s1 = ap_ptr[row + 1];
    for (int s = ap_ptr[row]; s < s1; ++s) {
        const int c = ap_col[s];
        const C<T>* v = ap_val + 16 * (int64_t)s + 4 * p;
        const C<T> a0 = v[0], a1 = v[1], a2 = v[2], a3 = v[3];
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            const C<T>* ev = e + (int64_t)(r0 + q) * lde + 4 * (int64_t)c;
            cfma(acc[q], a0, ev[0]);
            cfma(acc[q], a1, ev[1]);
            cfma(acc[q], a2, ev[2]);
            cfma(acc[q], a3, ev[3]);
        }
    }
#pragma unroll
    for (int q = 0; q < KT; ++q)
        if (!active || active[r0 + q]) {
            C<T>& o = t[(int64_t)(r0 + q) * ldt + d];
            o = csub(o, acc[q]);
        }
}

__global__ void k_finest_weights(const double* __restrict__ t, const uint8_t* __restrict__ fixmask, int64_t N,
                                 double* __restrict__ w) {
    const int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (d >= 4 * N) return;
    const int p = (int)(d & 3);
    const bool fixed = (fixmask[d >> 2] >> p) & 1u;
    w[d] = fixed ? 0.0 : 1.0 / t[d];
}

__global__ void k_d2f_real(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) b[e] = (float)a[e];
}

// scatter BSR blocks into a dense row-major nc x nc matrix
__global__ void k_densify(const int32_t* __restrict__ crow_of_slot, const int32_t* __restrict__ ccol,
                          const double2* __restrict__ cval, int64_t nnzc, int64_t nc, double2* __restrict__ dense) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= 16 * nnzc) return;
    const int64_t s = e >> 4;
    const int p = (int)((e >> 2) & 3), q = (int)(e & 3);
    dense[(4 * (int64_t)crow_of_slot[s] + p) * nc + 4 * (int64_t)ccol[s] + q] = cval[e];
}

}  // namespace

struct MgLevel {
    int64_t n = 0, nnzb = 0, n_agg = 0, n_next = 0;
    int max_agg = 0;
    const int32_t* rp = nullptr;
    const int32_t* col = nullptr;
    const double2* val64 = nullptr;
    const float2* val32 = nullptr;
    const float4* val32p = nullptr;          // FP32 values in the staged SpMM's row-pair layout
    DevBuf rp_own, col_own, val_own, val32_own, val32p_own;
    std::vector<int32_t> h_rp, h_col, h_agg_ptr;
    std::vector<uint8_t> h_free;             // 4n: unknown carries a near-null weight
    const int32_t* d_agg_ptr = nullptr;
    const int64_t* d_pinv_off = nullptr;
    const int64_t* d_pinv32_off = nullptr;   // packed FP32 inverses
    const double2* d_pinv64 = nullptr;
    const float2* d_pinv32 = nullptr;
    DevBuf agg_ptr_own, pinv_off_own, pinv32_off_own, pinv64_own, pinv32_own;
    DevBuf node_agg, clo, chi, w64, w32;
    DevBuf ap_ptr, ap_col, ap_val64, ap_val32, ap_val32p;  // AP = A P (this level's rows, next level's columns)
    std::vector<int32_t> h_ap_ptr, h_ap_col;
    bool has_ap = false;
    StagedPlan plan, ap_plan;                // staged FP32 SpMM tilings of A (levels > 0) and AP
    DevBuf r, z, t;                          // cycle vectors (k right-hand sides)
};

struct Multigrid {
    std::deque<MgLevel> L;                   // all levels but the coarsest (stable references)
    int64_t nc = 0;                          // unknowns of the coarsest level
    DevBuf einv64, einv32, rc, zc, gpart;
    int64_t kcap = 0;
    bool f32 = false;
    const StagedPlan* fine_plan = nullptr;   // the context's plan of the finest pattern
    const float2* val32t = nullptr;          // transposed FP32 blocks of the finest matrix
    int staged_rows = -1;                    // rows per staged tile the level plans were built for
};

void mg_free(Matrix& M) {
    delete M.mg;
    M.mg = nullptr;
}

namespace {

template <typename T>
const C<T>* lvl_pinv(const MgLevel& L);
template <>
const double2* lvl_pinv<double>(const MgLevel& L) { return L.d_pinv64; }
template <>
const float2* lvl_pinv<float>(const MgLevel& L) { return L.d_pinv32; }
template <typename T>
const int64_t* lvl_poff(const MgLevel& L);
template <>
const int64_t* lvl_poff<double>(const MgLevel& L) { return L.d_pinv_off; }
template <>
const int64_t* lvl_poff<float>(const MgLevel& L) { return L.d_pinv32_off; }
template <typename T>
const C<T>* lvl_val(const MgLevel& L);
template <>
const double2* lvl_val<double>(const MgLevel& L) { return L.val64; }
template <>
const float2* lvl_val<float>(const MgLevel& L) { return L.val32; }
template <typename T>
const T* lvl_w(const MgLevel& L);
template <>
const double* lvl_w<double>(const MgLevel& L) { return L.w64.as<double>(); }
template <>
const float* lvl_w<float>(const MgLevel& L) { return L.w32.as<float>(); }

void level_smoother(cudaStream_t st, MgLevel& L, bool f32) {
    // block inverses of the level's matrix over its (contiguous) aggregates
    const int64_t na = (int64_t)L.h_agg_ptr.size() - 1;
    L.n_agg = na;
    std::vector<int64_t> poff(na + 1, 0), poff32(na + 1, 0);
    int mx = 0;
    for (int64_t a = 0; a < na; ++a) {
        const int sz = L.h_agg_ptr[a + 1] - L.h_agg_ptr[a];
        mx = std::max(mx, sz);
        poff[a + 1] = poff[a] + (int64_t)(4 * sz) * (4 * sz);
        poff32[a + 1] = poff32[a] + sym_packed_size(4 * sz);
    }
    L.max_agg = mx;
    L.agg_ptr_own.alloc(sizeof(int32_t) * (na + 1));
    L.pinv_off_own.alloc(sizeof(int64_t) * (na + 1));
    ECT_CUDA(cudaMemcpyAsync(L.agg_ptr_own.p, L.h_agg_ptr.data(), L.agg_ptr_own.bytes, cudaMemcpyHostToDevice, st));
    ECT_CUDA(cudaMemcpyAsync(L.pinv_off_own.p, poff.data(), L.pinv_off_own.bytes, cudaMemcpyHostToDevice, st));
    L.pinv32_off_own.alloc(sizeof(int64_t) * (na + 1));
    ECT_CUDA(cudaMemcpyAsync(L.pinv32_off_own.p, poff32.data(), L.pinv32_off_own.bytes, cudaMemcpyHostToDevice, st));
    L.pinv64_own.alloc(sizeof(double2) * poff.back());
    if (f32) L.pinv32_own.alloc(sizeof(float2) * poff32.back());
    block_inverses(st, L.rp, L.col, L.val64, L.agg_ptr_own.as<int32_t>(), L.pinv_off_own.as<int64_t>(),
                   L.pinv32_off_own.as<int64_t>(), na, mx, L.pinv64_own.as<double2>(),
                   f32 ? L.pinv32_own.as<float2>() : nullptr);
    L.d_agg_ptr = L.agg_ptr_own.as<int32_t>();
    L.d_pinv_off = L.pinv_off_own.as<int64_t>();
    L.d_pinv32_off = L.pinv32_off_own.as<int64_t>();
    L.d_pinv64 = L.pinv64_own.as<double2>();
    L.d_pinv32 = f32 ? L.pinv32_own.as<float2>() : nullptr;
}

template <typename T>
void to_device(DevBuf& b, const std::vector<T>& h, cudaStream_t st) {
    b.alloc(sizeof(T) * std::max<size_t>(h.size(), 1));
    if (!h.empty()) ECT_CUDA(cudaMemcpyAsync(b.p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st));
}

// pattern of AP on the host (fine row i: the coarse nodes of its columns,
// ascending), values on the device
void build_ap(cudaStream_t st, MgLevel& L, const std::vector<int32_t>& nagg, bool f32) {
    const int64_t n = L.n;
    std::vector<int32_t> ptr(n + 1, 0), col, slot(L.nnzb);
    col.reserve((size_t)n * 6);
    std::vector<int32_t> row;
    for (int64_t i = 0; i < n; ++i) {
        row.clear();
        for (int32_t s = L.h_rp[i]; s < L.h_rp[i + 1]; ++s) row.push_back(nagg[L.h_col[s]]);
        std::sort(row.begin(), row.end());
        row.erase(std::unique(row.begin(), row.end()), row.end());
        const int32_t base = (int32_t)col.size();
        col.insert(col.end(), row.begin(), row.end());
        for (int32_t s = L.h_rp[i]; s < L.h_rp[i + 1]; ++s)
            slot[s] = base + (int32_t)(std::lower_bound(row.begin(), row.end(), nagg[L.h_col[s]]) - row.begin());
        ptr[i + 1] = (int32_t)col.size();
    }
    const int64_t nnz = (int64_t)col.size();
    std::vector<int32_t> sptr(nnz + 1, 0), src(L.nnzb);
    for (int64_t s = 0; s < L.nnzb; ++s) ++sptr[slot[s] + 1];
    for (int64_t b = 0; b < nnz; ++b) sptr[b + 1] += sptr[b];
    {
        std::vector<int32_t> fill(sptr.begin(), sptr.end() - 1);
        for (int64_t s = 0; s < L.nnzb; ++s) src[fill[slot[s]]++] = (int32_t)s;
    }
    DevBuf d_sptr, d_src;
    to_device(L.ap_ptr, ptr, st);
    to_device(L.ap_col, col, st);
    L.h_ap_ptr = ptr;
    L.h_ap_col = col;
    to_device(d_sptr, sptr, st);
    to_device(d_src, src, st);
    L.ap_val64.alloc(sizeof(double2) * 16 * std::max<int64_t>(nnz, 1));
    k_ap_values<<<grid_for(nnz, 128), 128, 0, st>>>(d_sptr.as<int32_t>(), d_src.as<int32_t>(), L.col, L.val64,
                                                     L.w64.as<double>(), nnz, L.ap_val64.as<double2>());
    ECT_CHECK_LAUNCH();
    if (f32) {
        L.ap_val32.alloc(sizeof(float2) * 16 * std::max<int64_t>(nnz, 1));
        to_f32(st, L.ap_val64.as<double2>(), L.ap_val32.as<float2>(), 16 * nnz);
        L.ap_val32p.alloc(sizeof(float2) * 16 * std::max<int64_t>(nnz, 1));
        to_pair_layout(st, L.ap_val32.as<float2>(), L.ap_val32p.as<float4>(), nnz);
    }
    ECT_CUDA(cudaStreamSynchronize(st));  // the host arrays above go out of scope
    L.has_ap = true;
}

template <typename T>
const C<T>* lvl_ap(const MgLevel& L);
template <>
const double2* lvl_ap<double>(const MgLevel& L) { return L.ap_val64.as<double2>(); }
template <>
const float2* lvl_ap<float>(const MgLevel& L) { return L.ap_val32.as<float2>(); }

template <typename T>
void ap_update(cudaStream_t st, const MgLevel& L, const C<T>* e, int64_t lde, C<T>* t, int64_t ldt, int k, int tile,
               const int* active) {
    const C<T>* val = lvl_ap<T>(L);
    const int32_t* ptr = L.ap_ptr.as<int32_t>();
    const int32_t* col = L.ap_col.as<int32_t>();
    for_tiles(k, tile, [&](int kt, int r, int nt) {
        const unsigned grid = tile_grid(grid_for(4 * L.n, 256), nt);
        const C<T>* er = e + r * lde;
        C<T>* tr = t + r * ldt;
        const int* ar = active ? active + r : nullptr;
        switch (kt) {
            case 8: k_ap_update<T, 8><<<grid, 256, 0, st>>>(ptr, col, val, er, lde, tr, ldt, L.n, ar, nt); break;
            case 4: k_ap_update<T, 4><<<grid, 256, 0, st>>>(ptr, col, val, er, lde, tr, ldt, L.n, ar, nt); break;
            case 2: k_ap_update<T, 2><<<grid, 256, 0, st>>>(ptr, col, val, er, lde, tr, ldt, L.n, ar, nt); break;
            default: k_ap_update<T, 1><<<grid, 256, 0, st>>>(ptr, col, val, er, lde, tr, ldt, L.n, ar, nt); break;
        }
    });
}

}  // namespace

void mg_setup(ect_ctx* c, int which, bool f32) {
    Matrix& M = ctx_mat(c, which);
    mg_free(M);
    cudaStream_t st = c->stream;
    Multigrid* G = new Multigrid();
    M.mg = G;
    G->f32 = f32;
    // ---- finest level: the matrix, its subdomain blocks and their inverses
    G->L.emplace_back();
    {
        MgLevel& L = G->L.back();
        L.n = c->n_nodes;
        L.nnzb = c->nnzb;
        L.rp = c->row_ptr.as<int32_t>();
        L.col = c->col.as<int32_t>();
        L.val64 = M.sval.as<double2>();
        L.val32 = f32 ? M.sval32.as<float2>() : nullptr;
        L.val32p = f32 ? M.sval32p.as<float4>() : nullptr;
        L.h_rp = c->h_row_ptr;
        L.h_col = c->h_col;
        L.h_agg_ptr = c->h_block_ptr;
        L.n_agg = c->n_blocks;
        L.max_agg = c->max_block_nodes;
        L.d_agg_ptr = c->block_ptr.as<int32_t>();
        L.d_pinv_off = c->pinv_off.as<int64_t>();
        L.d_pinv32_off = c->pinv_off32.as<int64_t>();
        L.d_pinv64 = M.pinv.as<double2>();
        L.d_pinv32 = f32 ? M.pinv32.as<float2>() : nullptr;
        L.h_free.resize(4 * L.n);
        for (int64_t i = 0; i < L.n; ++i)
            for (int p = 0; p < 4; ++p)
                L.h_free[4 * i + p] = !((M.h_fix[i] >> p) & 1);
        L.w64.alloc(sizeof(double) * 4 * L.n);
        k_finest_weights<<<grid_for(4 * L.n, 256), 256, 0, st>>>(M.t.as<double>(), M.fixmask.as<uint8_t>(), L.n,
                                                                 L.w64.as<double>());
        ECT_CHECK_LAUNCH();
        if (f32) {
            L.w32.alloc(sizeof(float) * 4 * L.n);
            k_d2f_real<<<grid_for(4 * L.n, 256), 256, 0, st>>>(L.w64.as<double>(), L.w32.as<float>(), 4 * L.n);
        }
    }
    // ---- coarsen until the coarse level has at most MAX_COARSE_DOFS unknowns
    for (int depth = 0; depth < 32; ++depth) {
        MgLevel& L = G->L.back();
        const int64_t n = L.n, na = (int64_t)L.h_agg_ptr.size() - 1;
        std::vector<int32_t> agg(n);
        for (int64_t a = 0; a < na; ++a)
            for (int32_t i = L.h_agg_ptr[a]; i < L.h_agg_ptr[a + 1]; ++i) agg[i] = (int32_t)a;
        // provisional coarse pattern (coarse node = aggregate index) and empty unknowns
        std::vector<std::vector<int32_t>> crow(na);
        std::vector<uint8_t> empty(4 * na, 1);
        for (int64_t a = 0; a < na; ++a) {
            std::vector<int32_t>& cr = crow[a];
            for (int32_t i = L.h_agg_ptr[a]; i < L.h_agg_ptr[a + 1]; ++i) {
                for (int p = 0; p < 4; ++p)
                    if (L.h_free[4 * i + p]) empty[4 * a + p] = 0;
                for (int32_t s = L.h_rp[i]; s < L.h_rp[i + 1]; ++s) cr.push_back(agg[L.h_col[s]]);
            }
            std::sort(cr.begin(), cr.end());
            cr.erase(std::unique(cr.begin(), cr.end()), cr.end());
        }
        const bool coarsest = 4 * na <= MAX_COARSE_DOFS;
        // aggregation of the coarse graph and renumbering (aggregates contiguous)
        std::vector<int32_t> cagg(na, -1), order(na), newid(na);
        if (coarsest) {
            std::iota(order.begin(), order.end(), 0);
        } else {
            int32_t nca = 0;
            for (int64_t I = 0; I < na; ++I) {
                if (cagg[I] >= 0) continue;
                int members = 1;
                cagg[I] = nca;
                for (int32_t J : crow[I]) {
                    if (members >= AGG_SIZE) break;
                    if (J != I && cagg[J] < 0) {
                        cagg[J] = nca;
                        ++members;
                    }
                }
                ++nca;
            }
            std::iota(order.begin(), order.end(), 0);
            std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cagg[a] < cagg[b]; });
        }
        for (int64_t k = 0; k < na; ++k) newid[order[k]] = (int32_t)k;
        // final coarse pattern in the new numbering
        std::vector<int32_t> nrp(na + 1, 0), ncol, ncrow;
        for (int64_t k = 0; k < na; ++k) {
            std::vector<int32_t> cols;
            for (int32_t J : crow[order[k]]) cols.push_back(newid[J]);
            std::sort(cols.begin(), cols.end());
            for (int32_t J : cols) {
                ncol.push_back(J);
                ncrow.push_back((int32_t)k);
            }
            nrp[k + 1] = (int32_t)ncol.size();
        }
        const int64_t nnzc = (int64_t)ncol.size();
        std::vector<uint8_t> nempty(4 * na);
        for (int64_t k = 0; k < na; ++k)
            for (int p = 0; p < 4; ++p) nempty[4 * k + p] = empty[4 * order[k] + p];
        // fine block -> coarse block map, then the per-coarse-block lists (fine blocks ascending)
        std::vector<int32_t> cslot(L.nnzb), frow(L.nnzb);
        for (int64_t i = 0; i < n; ++i) {
            const int32_t I = newid[agg[i]];
            const int32_t* b0 = ncol.data() + nrp[I];
            const int32_t* b1 = ncol.data() + nrp[I + 1];
            for (int32_t s = L.h_rp[i]; s < L.h_rp[i + 1]; ++s) {
                const int32_t J = newid[agg[L.h_col[s]]];
                cslot[s] = nrp[I] + (int32_t)(std::lower_bound(b0, b1, J) - b0);
                frow[s] = (int32_t)i;
            }
        }
        std::vector<int32_t> cptr(nnzc + 1, 0), clist(L.nnzb);
        for (int64_t s = 0; s < L.nnzb; ++s) ++cptr[cslot[s] + 1];
        for (int64_t q = 0; q < nnzc; ++q) cptr[q + 1] += cptr[q];
        {
            std::vector<int32_t> fill(cptr.begin(), cptr.end() - 1);
            for (int64_t s = 0; s < L.nnzb; ++s) clist[fill[cslot[s]]++] = (int32_t)s;
        }
        DevBuf d_cptr, d_clist, d_frow, d_crow, d_ccol, d_cempty, cval;
        to_device(d_cptr, cptr, st);
        to_device(d_clist, clist, st);
        to_device(d_frow, frow, st);
        to_device(d_crow, ncrow, st);
        to_device(d_ccol, ncol, st);
        to_device(d_cempty, nempty, st);
        cval.alloc(sizeof(double2) * 16 * std::max<int64_t>(nnzc, 1));
        k_galerkin<<<grid_for(nnzc, 128), 128, 0, st>>>(d_cptr.as<int32_t>(), d_clist.as<int32_t>(),
                                                         d_frow.as<int32_t>(), L.col, L.val64, L.w64.as<double>(),
                                                         nnzc, d_crow.as<int32_t>(), d_ccol.as<int32_t>(),
                                                         d_cempty.as<uint8_t>(), cval.as<double2>());
        ECT_CHECK_LAUNCH();
        // restriction / prolongation maps of this level
        std::vector<int32_t> nagg(n), lo(na), hi(na);
        for (int64_t i = 0; i < n; ++i) nagg[i] = newid[agg[i]];
        for (int64_t k = 0; k < na; ++k) {
            lo[k] = L.h_agg_ptr[order[k]];
            hi[k] = L.h_agg_ptr[order[k] + 1];
        }
        to_device(L.node_agg, nagg, st);
        to_device(L.clo, lo, st);
        to_device(L.chi, hi, st);
        L.n_next = na;
        if (L.n > WARP_ROW_MAX_NODES) build_ap(st, L, nagg, f32);  // small levels: latency-bound either way
        ECT_CUDA(cudaStreamSynchronize(st));
        if (coarsest) {
            const int64_t nc = 4 * na;
            G->nc = nc;
            G->einv64.alloc(sizeof(double2) * nc * nc);
            ECT_CUDA(cudaMemsetAsync(G->einv64.p, 0, G->einv64.bytes, st));
            k_densify<<<grid_for(16 * nnzc, 256), 256, 0, st>>>(d_crow.as<int32_t>(), d_ccol.as<int32_t>(),
                                                                cval.as<double2>(), nnzc, nc, G->einv64.as<double2>());
            ECT_CHECK_LAUNCH();
            dense_inverse(st, G->einv64.as<double2>(), nc);
            if (f32) {
                G->einv32.alloc(sizeof(float2) * nc * nc);
                to_f32(st, G->einv64.as<double2>(), G->einv32.as<float2>(), nc * nc);
            }
            ECT_CUDA(cudaStreamSynchronize(st));
            return;
        }
        // next level
        std::vector<int32_t> nagg_ptr(1, 0);
        for (int64_t k = 1; k <= na; ++k)
            if (k == na || cagg[order[k]] != cagg[order[k - 1]]) nagg_ptr.push_back((int32_t)k);
        G->L.emplace_back();
        MgLevel& Lc = G->L.back();
        Lc.n = na;
        Lc.nnzb = nnzc;
        Lc.h_rp = nrp;
        Lc.h_col = ncol;
        Lc.h_agg_ptr = nagg_ptr;
        to_device(Lc.rp_own, nrp, st);
        to_device(Lc.col_own, ncol, st);
        Lc.rp = Lc.rp_own.as<int32_t>();
        Lc.col = Lc.col_own.as<int32_t>();
        Lc.val_own.alloc(cval.bytes);
        ECT_CUDA(cudaMemcpyAsync(Lc.val_own.p, cval.p, cval.bytes, cudaMemcpyDeviceToDevice, st));
        Lc.val64 = Lc.val_own.as<double2>();
        if (f32) {
            Lc.val32_own.alloc(sizeof(float2) * 16 * nnzc);
            to_f32(st, Lc.val64, Lc.val32_own.as<float2>(), 16 * nnzc);
            Lc.val32 = Lc.val32_own.as<float2>();
            Lc.val32p_own.alloc(sizeof(float2) * 16 * std::max<int64_t>(nnzc, 1));
            to_pair_layout(st, Lc.val32, Lc.val32p_own.as<float4>(), nnzc);
            Lc.val32p = Lc.val32p_own.as<float4>();
        }
        Lc.h_free.resize(4 * na);
        std::vector<double> w(4 * na);
        std::vector<float> wf(4 * na);
        for (int64_t d = 0; d < 4 * na; ++d) {
            Lc.h_free[d] = !nempty[d];
            w[d] = nempty[d] ? 0.0 : 1.0;
            wf[d] = (float)w[d];
        }
        to_device(Lc.w64, w, st);
        to_device(Lc.w32, wf, st);
        level_smoother(st, Lc, f32);
        ECT_CUDA(cudaStreamSynchronize(st));
    }
    throw EctError{ECT_ERR_ARG, "multigrid did not reach the coarsest size"};
}

void mg_scratch(Matrix& M, int k) {
    Multigrid* G = M.mg;
    if (!G || G->kcap >= k) return;
    for (size_t l = 0; l < G->L.size(); ++l) {
        MgLevel& L = G->L[l];
        const size_t bytes = sizeof(double2) * 4 * (size_t)L.n * k;
        L.t.alloc(bytes);
        if (l > 0) {
            L.r.alloc(bytes);
            L.z.alloc(bytes);
        }
    }
    G->rc.alloc(sizeof(double2) * G->nc * k);
    G->zc.alloc(sizeof(double2) * G->nc * k);
    G->gpart.alloc(sizeof(double2) * gemv_scratch_elems(G->nc, k));
    G->kcap = k;
}

namespace {

template <typename T>
void cycle(cudaStream_t st, Multigrid* G, size_t l, const C<T>* r, C<T>* z, int k, int tile, const int* active) {
    if (l == G->L.size()) {
        const C<T>* e = std::is_same<T, double>::value ? (const C<T>*)G->einv64.p : (const C<T>*)G->einv32.p;
        dense_gemv<T>(st, e, G->nc, r, z, k, tile, active, (C<T>*)G->gpart.p);
        return;
    }
    MgLevel& L = G->L[l];
    const int64_t ld = 4 * L.n;
    const bool last = (l + 1 == G->L.size());
    const int64_t ldn = last ? G->nc : 4 * G->L[l + 1].n;
    C<T>* rn = last ? (C<T>*)G->rc.p : (C<T>*)G->L[l + 1].r.p;
    C<T>* zn = last ? (C<T>*)G->zc.p : (C<T>*)G->L[l + 1].z.p;
    C<T>* t = (C<T>*)L.t.p;
    const C<T>* val = lvl_val<T>(L);
    const T* w = lvl_w<T>(L);
    block_apply<T>(st, L.d_agg_ptr, lvl_poff<T>(L), lvl_pinv<T>(L), L.n_agg, L.max_agg, r, z, k, ld, tile, active,
                   false);
    const int gamma = last ? 1 : 2;
    // t = r - A z: one thread per scalar row, or one warp per block row on the small coarse
    // levels (few rows, many blocks per row: the warp splits the row's serial chain of loads)
    const StagedPlan* plan = l == 0 ? G->fine_plan : &L.plan;
    const bool staged = std::is_same<T, float>::value && G->staged_rows > 0 && plan && plan->ok;
    const bool colwarp = std::is_same<T, float>::value && G->staged_rows == SPMM_COLWARP && l == 0 && G->val32t;
    auto residual = [&]() {
        if (colwarp)
            bsr_spmm_colwarp_f32(st, L.rp, L.col, G->val32t, L.n, (const float2*)z, ld, (const float2*)r, (float2*)t,
                                 ld, k, active);
        else if (staged && L.n > WARP_ROW_MAX_NODES)
            bsr_spmm_staged_f32(st, *plan, L.rp, L.val32p, (const float2*)z, ld, (const float2*)r, (float2*)t, ld, k,
                                active);
        else if (L.n <= WARP_ROW_MAX_NODES)
            bsr_spmv_warp<T>(st, L.rp, L.col, val, L.n, z, r, t, k, ld, tile, active);
        else if (std::is_same<T, double>::value)
            bsr_spmv_f64(st, L.rp, L.col, (const double2*)val, L.n, (const double2*)z, (const double2*)r, (double2*)t,
                         k, ld, tile, active);
        else
            bsr_spmv_f32(st, L.rp, L.col, (const float2*)val, L.n, (const float2*)z, (const float2*)r, (float2*)t, k,
                         ld, tile, active);
    };
    // With AP the residual after each coarse correction is updated in place
    // (t -= AP e) instead of recomputed, so only the first one is a full SpMM.
    for (int g = 0; g < gamma; ++g) {
        if (g == 0 || !L.has_ap) residual();
        k_restrict<T><<<dim3(grid_for(4 * L.n_next, 256), k), 256, 0, st>>>(
            t, ld, L.clo.as<int32_t>(), L.chi.as<int32_t>(), w, L.n_next, k, active, rn, ldn);
        cycle<T>(st, G, l + 1, rn, zn, k, tile, active);
        k_prolong<T><<<dim3(grid_for(4 * L.n, 256), k), 256, 0, st>>>(z, ld, L.node_agg.as<int32_t>(), w, L.n, zn, ldn,
                                                                        active);
        if (L.has_ap) {
            if (std::is_same<T, float>::value && G->staged_rows > 0 && L.ap_plan.ok)
                bsr_spmm_staged_f32(st, L.ap_plan, L.ap_ptr.as<int32_t>(), L.ap_val32p.as<float4>(),
                                    (const float2*)zn, ldn, (const float2*)t, (float2*)t, ld, k, active);
            else
                ap_update<T>(st, L, zn, ldn, t, ld, k, tile, active);
        }
    }
    if (!L.has_ap) residual();
    block_apply<T>(st, L.d_agg_ptr, lvl_poff<T>(L), lvl_pinv<T>(L), L.n_agg, L.max_agg, t, z, k, ld, tile, active,
                   true);
    ECT_CHECK_LAUNCH();
}

}  // namespace

void mg_apply_f64(ect_ctx* c, int which, const double2* r, double2* z, int k, int64_t ld, int tile, const int* active) {
    Matrix& M = ctx_mat(c, which);
    ECT_REQUIRE(M.mg && M.mg->kcap >= k, ECT_ERR_STATE, "multigrid scratch not ready (internal)");
    ECT_REQUIRE(ld == 4 * c->n_nodes, ECT_ERR_ARG, "multigrid vectors must be packed");
    cycle<double>(c->stream, M.mg, 0, r, z, k, tile, active);
}

void mg_apply_f32(ect_ctx* c, int which, const float2* r, float2* z, int k, int64_t ld, int tile, const int* active) {
    Matrix& M = ctx_mat(c, which);
    ECT_REQUIRE(M.mg && M.mg->kcap >= k && M.mg->f32, ECT_ERR_STATE, "FP32 multigrid not ready");
    ECT_REQUIRE(ld == 4 * c->n_nodes, ECT_ERR_ARG, "multigrid vectors must be packed");
    cycle<float>(c->stream, M.mg, 0, r, z, k, tile, active);
}

void staged_prepare(ect_ctx* c, int which) {
    const int rows = c->staged_rows;
    Matrix& M = ctx_mat(c, which);
    Multigrid* G = M.mg;
    if (rows <= 0) {
        if (rows == SPMM_COLWARP && M.has_f32 && M.t_gen != M.val_gen) {  // transposed blocks, on demand
            if (!M.sval32t.p) M.sval32t.alloc(sizeof(float2) * 16 * c->nnzb);
            to_transposed_layout(c->stream, M.sval32.as<float2>(), M.sval32t.as<float2>(), c->nnzb);
            M.t_gen = M.val_gen;
        }
        if (G) {
            G->staged_rows = rows == SPMM_COLWARP ? SPMM_COLWARP : -1;
            G->val32t = rows == SPMM_COLWARP ? M.sval32t.as<float2>() : nullptr;
        }
        return;
    }
    cudaStream_t st = c->stream;
    if (c->fine_plan.rows != rows) {
        staged_plan_build(st, c->fine_plan, c->h_row_ptr, c->h_col, c->n_nodes, c->n_nodes, rows);
        ++c->plan_gen;
    }
    if (!G) return;
    G->fine_plan = &c->fine_plan;
    if (G->f32) {
        bool rebuilt = false;
        for (size_t l = 0; l < G->L.size(); ++l) {
            MgLevel& L = G->L[l];
            if (l > 0 && L.n > WARP_ROW_MAX_NODES && L.plan.rows != rows) {
                staged_plan_build(st, L.plan, L.h_rp, L.h_col, L.n, L.n, rows);
                rebuilt = true;
            }
            if (L.has_ap && L.ap_plan.rows != rows) {
                staged_plan_build(st, L.ap_plan, L.h_ap_ptr, L.h_ap_col, L.n, L.n_next, rows);
                rebuilt = true;
            }
        }
        if (rebuilt) ++c->plan_gen;
    }
    G->staged_rows = rows;
}

int mg_levels(const Matrix& M) { return M.mg ? (int)M.mg->L.size() + 1 : 0; }

bool mg_ready(const Matrix& M, int k) { return M.mg && M.mg->kcap >= k; }
