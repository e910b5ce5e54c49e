// Kernel (b), staged form: BSR (4x4 complex FP32 blocks) SpMM for up to 8
// right-hand sides per work item, with the operands staged in shared memory
// by a persistent, software-pipelined CTA per SM.
//
// The rows of the matrix are cut into tiles of consecutive block rows (the
// subdomain-major node order makes a tile a compact piece of the mesh).  For
// each tile the plan holds its metadata record (the row offsets and, per
// block, the position of the block's column node in the tile's column list)
// and the column list itself, which covers the tile's distinct column nodes
// with runs of consecutive nodes.  A work item is (tile, tile of 8 right-hand
// sides).  Each CTA walks the items b, b + G, b + 2G, ... through a ring of S
// shared-memory stages, S - 1 items ahead of the one it computes:
//   * one thread starts two bulk copies (TMA engine) per item: the tile's
//     blocks (a contiguous nnz_tile x 128 bytes) and its metadata record,
//     completing on the stage's mbarrier;
//   * every thread copies the x values of one (column node, half) of the list
//     for the 8 right-hand sides with 16-byte asynchronous copies (x is laid
//     out [rhs q][column][4 complex] in the stage; list entries are mostly
//     consecutive nodes, so a warp's copies are contiguous runs); the node
//     index is loaded one item earlier still, so no copy waits for it;
//   * compute: one warp per block row; lane (p, q) owns scalar row p of
//     right-hand side q, reads row p of each block and the 4 values of x_q at
//     the block's column node from shared memory (conflict-free), keeps one
//     complex accumulator and stores y (or b - A x) directly.
// The matrix streams from HBM while earlier stages are being computed, every
// x value of a tile's list is read once per item, and no gather goes through
// L1.  The mbarrier wait is bounded: on expiry the CTA sets a device flag
// (read by staged_take_error) and leaves.
#include <algorithm>
#include <numeric>

#include "common.cuh"
#include "tc05.cuh"

namespace {

constexpr int STG_KT = 8;                // right-hand sides per work item
constexpr int STG_WARPS = 16;
constexpr int STG_THREADS = 32 * STG_WARPS;
constexpr int MAX_STAGES = 4;
constexpr int MAX_TILE_ROWS = 64;
constexpr int MAX_TILE_BLOCKS = 512;
constexpr int MAX_TILE_COLS = STG_THREADS / 2;  // one (column, half) per thread
constexpr int STG_SMEM_MAX = 232448;     // dynamic shared memory a CTA may use (227 KB)
constexpr uint32_t STG_WAIT = 1u << 22;  // bounded polls of an mbarrier

__device__ int g_staged_err = 0;

struct StageLayout {
    uint32_t mat, meta, x, xq, stage;  // byte offsets inside a stage, x stride per rhs, stage size
    int stages;
};

inline int round_up(int v, int a) { return (v + a - 1) / a * a; }

// one stage: blocks | metadata record | x window [rhs q][column][4 complex]; the stride of
// a right-hand side is 16 bytes past a multiple of 128, so the 8 lane groups q that read
// the same column hit 8 different bank groups
inline StageLayout stage_layout(int max_blocks, int max_meta, int max_cols) {
    StageLayout L;
    L.mat = 0;
    L.meta = (uint32_t)max_blocks * 128;
    L.x = L.meta + (uint32_t)round_up(max_meta, 128);
    L.xq = (uint32_t)round_up(max_cols * 32, 128) + 16;
    L.stage = (uint32_t)round_up((int)(L.x + STG_KT * L.xq), 128);
    L.stages = std::min<int>(MAX_STAGES, (STG_SMEM_MAX - 128) / (int)L.stage);
    return L;
}

__device__ __forceinline__ bool bwait(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < STG_WAIT; ++i)
        if (tc05::mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void cfma4(float2& acc, const float4& a01, const float4& a23, const float4& x01,
                                      const float4& x23) {
    cfma(acc, make_float2(a01.x, a01.y), make_float2(x01.x, x01.y));
    cfma(acc, make_float2(a01.z, a01.w), make_float2(x01.z, x01.w));
    cfma(acc, make_float2(a23.x, a23.y), make_float2(x23.x, x23.y));
    cfma(acc, make_float2(a23.z, a23.w), make_float2(x23.z, x23.w));
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc05::smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

struct PipeArgs {
    const int32_t* rp;
    const int32_t* tile_row;
    const int32_t* tile_cptr;
    const int32_t* meta_off;
    const uint8_t* meta;
    const int32_t* cols;
    const float2* val;
    const float2* x;
    int64_t ldx;
    const float2* b;
    float2* y;
    int64_t ldy;
    const int* active;
    int k, nrt;
    int64_t n_items;
    uint32_t off_meta, off_x, xq, stage_bytes;
};

// the column node this thread copies for item `item` (-1: none)
__device__ __forceinline__ int item_col(const PipeArgs& a, int64_t item) {
    if (item >= a.n_items) return -1;
    const int tile = (int)(item / a.nrt);
    const int c0 = a.tile_cptr[tile], nc = a.tile_cptr[tile + 1] - c0;
    const int cl = threadIdx.x >> 1;
    return cl < nc ? a.cols[c0 + cl] : -1;
}

// stage `item` into `st`: bulk copies of blocks and metadata (thread 0) and the
// x values of this thread's (column, half) for the item's right-hand sides
__device__ __forceinline__ void stage_item(const PipeArgs& a, int64_t item, int node, unsigned char* st,
                                           uint64_t* full) {
    if (item >= a.n_items) return;
    const int tile = (int)(item / a.nrt), r0 = (int)(item % a.nrt) * STG_KT;
    const int kt = min(STG_KT, a.k - r0);
    if (threadIdx.x == 0) {
        const int row0 = a.tile_row[tile], row1 = a.tile_row[tile + 1];
        const int blk0 = a.rp[row0], blk1 = a.rp[row1];
        const int mo0 = a.meta_off[tile], mo1 = a.meta_off[tile + 1];
        const uint32_t mbytes = (uint32_t)(blk1 - blk0) * 128u, tbytes = (uint32_t)(mo1 - mo0) * 16u;
        tc05::mbar_expect_tx(full, mbytes + tbytes);
        tc05::bulk_g2s(st, a.val + 16 * (int64_t)blk0, mbytes, full);
        tc05::bulk_g2s(st + a.off_meta, a.meta + 16 * (int64_t)mo0, tbytes, full);
    }
    if (node >= 0) {
        const int cl = threadIdx.x >> 1, h = threadIdx.x & 1;
        unsigned char* dst = st + a.off_x + (uint32_t)cl * 32u + (uint32_t)h * 16u;
        const float2* src = a.x + (int64_t)r0 * a.ldx + 4 * (int64_t)node + 2 * h;
        for (int q = 0; q < kt; ++q) cp_async16(dst + (uint32_t)q * a.xq, src + (int64_t)q * a.ldx);
    }
}

template <int S>
__global__ void __launch_bounds__(STG_THREADS, 1) k_spmm_pipe(const PipeArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    unsigned char* base = smem + 128;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, p = lane & 3, q = lane >> 2;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) tc05::mbar_init(&full[s], 1);
        tc05::fence_barrier_init();
    }
    __syncthreads();
    const int64_t G = gridDim.x, b0 = blockIdx.x;
    // prologue: items 0 .. S-2 of this CTA into stages 0 .. S-2
    for (int j = 0; j < S - 1; ++j) {
        const int64_t item = b0 + j * G;
        stage_item(a, item, item_col(a, item), base + (size_t)j * a.stage_bytes, &full[j]);
        cp_async_commit();
    }
    int next_col = item_col(a, b0 + (S - 1) * G);
    for (int64_t j = 0;; ++j) {
        const int64_t item = b0 + j * G;
        if (item >= a.n_items) break;
        const int s = (int)(j % S);
        __syncthreads();  // every warp is done with item j - 1: its stage takes item j + S - 1
        {
            const int64_t ahead = item + (S - 1) * G;
            const int sa = (int)((j + S - 1) % S);
            stage_item(a, ahead, next_col, base + (size_t)sa * a.stage_bytes, &full[sa]);
            cp_async_commit();
            next_col = item_col(a, ahead + G);
        }
        cp_async_wait<S - 1>();  // this thread's copies for item j have landed
        __syncthreads();         // ... and everyone else's
        if (!bwait(&full[s], (uint32_t)(j / S) & 1u)) {
            if (threadIdx.x == 0) atomicOr(&g_staged_err, 1);
            cp_async_wait<0>();
            return;
        }
        const unsigned char* st = base + (size_t)s * a.stage_bytes;
        const int tile = (int)(item / a.nrt), r0 = (int)(item % a.nrt) * STG_KT;
        const int kt = min(STG_KT, a.k - r0);
        const bool store = q < kt && (!a.active || a.active[r0 + q]);
        const int row0 = a.tile_row[tile], row1 = a.tile_row[tile + 1];
        const int32_t* rps = reinterpret_cast<const int32_t*>(st + a.off_meta);
        const uint16_t* lcs = reinterpret_cast<const uint16_t*>(rps + (row1 - row0 + 1));
        const float4* ms4 = reinterpret_cast<const float4*>(st);
        const unsigned char* xq = st + a.off_x + (uint32_t)q * a.xq;
        for (int i = row0 + warp; i < row1; i += STG_WARPS) {
            const int64_t e = (int64_t)(r0 + q) * a.ldy + 4 * (int64_t)i + p;
            const float2 bv = (a.b && store) ? a.b[e] : make_float2(0.f, 0.f);  // in flight during the row
            const int s0 = rps[i - row0], s1 = rps[i - row0 + 1];
            float2 acc = make_float2(0.f, 0.f), acc2 = make_float2(0.f, 0.f);
            for (int sb = s0; sb < s1; sb += 32) {
                const int n = min(32, s1 - sb);
                const int lcv = lane < n ? (int)lcs[sb + lane] : 0;
                const float4* mrow = ms4 + (int64_t)sb * 8 + 2 * p;
                int jj = 0;
                for (; jj + 1 < n; jj += 2) {
                    const int l0 = __shfl_sync(0xffffffffu, lcv, jj);
                    const int l1 = __shfl_sync(0xffffffffu, lcv, jj + 1);
                    const float4* x0 = reinterpret_cast<const float4*>(xq + (uint32_t)l0 * 32u);
                    const float4* x1 = reinterpret_cast<const float4*>(xq + (uint32_t)l1 * 32u);
                    const float4 a01 = mrow[8 * jj], a23 = mrow[8 * jj + 1];
                    const float4 b01 = mrow[8 * jj + 8], b23 = mrow[8 * jj + 9];
                    const float4 u01 = x0[0], u23 = x0[1], v01 = x1[0], v23 = x1[1];
                    cfma4(acc, a01, a23, u01, u23);
                    cfma4(acc2, b01, b23, v01, v23);
                }
                if (jj < n) {
                    const int l0 = __shfl_sync(0xffffffffu, lcv, jj);
                    const float4* x0 = reinterpret_cast<const float4*>(xq + (uint32_t)l0 * 32u);
                    cfma4(acc, mrow[8 * jj], mrow[8 * jj + 1], x0[0], x0[1]);
                }
            }
            acc.x += acc2.x;
            acc.y += acc2.y;
            if (store) a.y[e] = a.b ? csub(bv, acc) : acc;
        }
    }
    cp_async_wait<0>();  // nothing of this CTA's may still be in flight when it leaves
}

}  // namespace


// Tiles of at most `rows` consecutive block rows (and MAX_TILE_BLOCKS blocks).
// A tile's column list covers its distinct column nodes with runs of
// consecutive nodes; two runs are merged when the gap between them is at
// most RUN_GAP nodes (a few unneeded x values in exchange for longer
// contiguous copies).  The list holds at most MAX_TILE_COLS nodes (a tile is
// shortened until it does).
constexpr int RUN_GAP = 4;

namespace {

// covering list of the distinct columns of blocks [s0, s1); returns its length
int cover(const std::vector<int32_t>& col, int32_t s0, int32_t s1, std::vector<int32_t>& cols,
          std::vector<int32_t>& list) {
    cols.assign(col.begin() + s0, col.begin() + s1);
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
    list.clear();
    size_t u = 0;
    while (u < cols.size()) {
        size_t v = u;
        while (v + 1 < cols.size() && cols[v + 1] - cols[v] - 1 <= RUN_GAP) ++v;
        for (int32_t c = cols[u]; c <= cols[v]; ++c) list.push_back(c);
        u = v + 1;
    }
    return (int)list.size();
}

}  // namespace

void staged_plan_build(cudaStream_t st, StagedPlan& P, const std::vector<int32_t>& rp,
                       const std::vector<int32_t>& col, int64_t n_rows, int64_t n_cols, int rows) {
    P.reset();
    P.rows = rows;
    P.n_rows = n_rows;
    if (n_rows == 0 || rows <= 0) return;
    const int rmax = std::min(rows, MAX_TILE_ROWS);
    std::vector<int32_t> trow(1, 0), tcptr(1, 0), moff(1, 0), tcols;
    std::vector<uint8_t> meta;
    std::vector<int32_t> cols, list, loc(n_cols, 0);
    int64_t i = 0;
    while (i < n_rows) {
        int64_t e = i;
        int64_t blocks = 0;
        while (e < n_rows && e - i < rmax && blocks + (rp[e + 1] - rp[e]) <= MAX_TILE_BLOCKS) {
            blocks += rp[e + 1] - rp[e];
            ++e;
        }
        if (e == i) return;  // one row alone exceeds the block limit: no plan
        int nc = cover(col, rp[i], rp[e], cols, list);
        while (nc > MAX_TILE_COLS && e > i + 1) {  // shorten the tile until its list fits
            --e;
            nc = cover(col, rp[i], rp[e], cols, list);
        }
        if (nc > MAX_TILE_COLS) return;
        blocks = rp[e] - rp[i];
        for (int u = 0; u < nc; ++u) loc[list[u]] = u;
        // metadata record: row offsets (int32) then local columns (uint16), padded to 16 bytes
        const size_t m0 = meta.size();
        const int64_t nr = e - i;
        const size_t bytes = (size_t)(nr + 1) * 4 + (size_t)blocks * 2;
        meta.resize(m0 + (bytes + 15) / 16 * 16, 0);
        int32_t* ro = reinterpret_cast<int32_t*>(meta.data() + m0);
        uint16_t* lc = reinterpret_cast<uint16_t*>(meta.data() + m0 + (size_t)(nr + 1) * 4);
        for (int64_t r = 0; r <= nr; ++r) ro[r] = rp[i + r] - rp[i];
        for (int32_t s = rp[i]; s < rp[e]; ++s) lc[s - rp[i]] = (uint16_t)loc[col[s]];
        tcols.insert(tcols.end(), list.begin(), list.end());
        P.max_blocks = std::max<int>(P.max_blocks, (int)blocks);
        P.max_cols = std::max<int>(P.max_cols, nc);
        P.max_meta = std::max<int>(P.max_meta, (int)(meta.size() - m0));
        trow.push_back((int32_t)e);
        tcptr.push_back((int32_t)tcols.size());
        moff.push_back((int32_t)(meta.size() / 16));
        i = e;
    }
    P.n_tiles = (int64_t)trow.size() - 1;
    const StageLayout L = stage_layout(P.max_blocks, P.max_meta, P.max_cols);
    if (L.stages < 2) return;  // tiles too large for a double-buffered ring
    ECT_REQUIRE(tcols.size() < (1ull << 31) && meta.size() / 16 < (1ull << 31), ECT_ERR_ARG,
                "staged SpMM plan too large (internal)");
    auto up = [&](DevBuf& d, const void* h, size_t bytes) {
        d.alloc(std::max<size_t>(bytes, 16));
        if (bytes) ECT_CUDA(cudaMemcpyAsync(d.p, h, bytes, cudaMemcpyHostToDevice, st));
    };
    up(P.tile_row, trow.data(), sizeof(int32_t) * trow.size());
    up(P.tile_cptr, tcptr.data(), sizeof(int32_t) * tcptr.size());
    up(P.tile_meta_off, moff.data(), sizeof(int32_t) * moff.size());
    up(P.tile_meta, meta.data(), meta.size());
    up(P.tile_cols, tcols.data(), sizeof(int32_t) * tcols.size());
    ECT_CUDA(cudaFuncSetAttribute(k_spmm_pipe<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, STG_SMEM_MAX));
    ECT_CUDA(cudaFuncSetAttribute(k_spmm_pipe<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, STG_SMEM_MAX));
    ECT_CUDA(cudaFuncSetAttribute(k_spmm_pipe<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, STG_SMEM_MAX));
    ECT_CUDA(cudaStreamSynchronize(st));  // the host vectors go out of scope
    P.ok = true;
}

void bsr_spmm_staged_f32(cudaStream_t st, const StagedPlan& P, const int32_t* rp, const float2* val,
                         const float2* x, int64_t ldx, const float2* b, float2* y, int64_t ldy, int k,
                         const int* active) {
    ECT_REQUIRE(P.ok, ECT_ERR_STATE, "staged SpMM plan not built (internal)");
    if (P.n_tiles == 0 || k <= 0) return;
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        ECT_CUDA(cudaGetDevice(&dev));
        ECT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const StageLayout L = stage_layout(P.max_blocks, P.max_meta, P.max_cols);
    PipeArgs a;
    a.rp = rp;
    a.tile_row = P.tile_row.as<int32_t>();
    a.tile_cptr = P.tile_cptr.as<int32_t>();
    a.meta_off = P.tile_meta_off.as<int32_t>();
    a.meta = P.tile_meta.as<uint8_t>();
    a.cols = P.tile_cols.as<int32_t>();
    a.val = val;
    a.x = x;
    a.ldx = ldx;
    a.b = b;
    a.y = y;
    a.ldy = ldy;
    a.active = active;
    a.k = k;
    a.nrt = (k + STG_KT - 1) / STG_KT;
    a.n_items = P.n_tiles * a.nrt;
    a.off_meta = L.meta;
    a.off_x = L.x;
    a.xq = L.xq;
    a.stage_bytes = L.stage;
    const unsigned grid = (unsigned)std::min<int64_t>(a.n_items, (int64_t)sms);
    const size_t smem = 128 + (size_t)L.stages * L.stage;
    switch (L.stages) {
        case 2: k_spmm_pipe<2><<<grid, STG_THREADS, smem, st>>>(a); break;
        case 3: k_spmm_pipe<3><<<grid, STG_THREADS, smem, st>>>(a); break;
        default: k_spmm_pipe<4><<<grid, STG_THREADS, smem, st>>>(a); break;
    }
    ECT_CHECK_LAUNCH();
}

int staged_take_error(cudaStream_t st) {
    int h = 0;
    const int zero = 0;
    ECT_CUDA(cudaMemcpyFromSymbolAsync(&h, g_staged_err, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
    ECT_CUDA(cudaStreamSynchronize(st));
    if (h) ECT_CUDA(cudaMemcpyToSymbol(g_staged_err, &zero, sizeof(int)));
    return h;
}
