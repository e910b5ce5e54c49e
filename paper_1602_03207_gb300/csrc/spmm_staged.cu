// Kernel (b), staged form: BSR (4x4 complex FP32 blocks) SpMM for up to 8
// right-hand sides per work item, with the operands staged in shared memory
// by a persistent, warp-specialised pipeline (one CTA per SM).
//
// The rows of the matrix are cut into tiles of consecutive block rows (the
// subdomain-major node order makes a tile a compact piece of the mesh).  For
// each tile the plan holds its metadata record (its row range, the row
// offsets and, per block, the position of the block's column node in the
// tile's column list)
// and the column list itself, which covers the tile's distinct column nodes
// with runs of consecutive nodes.  A work item is (tile, tile of 8 right-hand
// sides).  Each CTA walks the items b, b + G, b + 2G, ... through a ring of S
// shared-memory stages:
//   * producer warps: once an item's stage is free, one thread starts two
//     bulk copies (TMA engine) of the tile's blocks (a contiguous nnz_tile x
//     128 bytes) and of its metadata record, and the producer threads copy
//     the x values of every (column node, half) of the list for the 8
//     right-hand sides with 16-byte asynchronous copies (x is laid out [rhs
//     q][column][4 complex] in the stage; list entries are mostly consecutive
//     nodes, so a warp's copies are contiguous runs); all of it completes on
//     the stage's "full" mbarrier;
//   * consumer warps: two block rows per warp, the half-warps on alternate
//     blocks of a row; lane (pp, qq) of an eight-lane group owns scalar rows
//     2pp, 2pp + 1 of right-hand sides 2qq, 2qq + 1,
//     reads those two rows of each block and the x values of its two right-
//     hand sides at the block's column node from shared memory (one 16-byte
//     load feeds two outputs), keeps four complex accumulators and stores y
//     (or b - A x) directly, then the warp arrives on the stage's "empty"
//     mbarrier.
// There is no CTA-wide barrier in the loop: the matrix streams from HBM while
// earlier stages are computed, every x value of a tile's list is read once
// per item, and no gather goes through L1.  All waits are bounded: on expiry
// a thread sets a device flag (read by staged_take_error) and leaves.
#include <algorithm>
#include <numeric>

#include "common.cuh"
#include "tc05.cuh"

namespace {

constexpr int STG_KT = 8;                // right-hand sides per work item
constexpr int PRODUCER_WARPS = 4;       // stage the next items
constexpr int CONSUMER_WARPS = 20;      // compute: two block rows per warp at a time
constexpr int STG_WARPS = PRODUCER_WARPS + CONSUMER_WARPS;
constexpr int STG_THREADS = 32 * STG_WARPS;
constexpr int PRODUCER_THREADS = 32 * PRODUCER_WARPS;
constexpr int MAX_STAGES = 4;
constexpr int MAX_TILE_ROWS = 64;
constexpr int MAX_TILE_BLOCKS = 512;
constexpr int PRODUCER_PAIRS = 4;       // (column, half) pairs per producer thread and item
constexpr int MAX_TILE_COLS = PRODUCER_PAIRS * PRODUCER_THREADS / 2;
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
    const float4* val;  // row-pair layout, 8 float4 per block
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

__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(tc05::smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc05::smem_addr(bar)) : "memory");
}

// Producer warps: for each item of this CTA, once its stage is free, thread 0
// starts the bulk copies of the tile's blocks and metadata (expected bytes on
// the stage's "full" mbarrier), and the producer threads copy x for every
// (column, half) of the tile's list and every right-hand side with 16-byte
// asynchronous copies whose completion also arrives on "full".  Consumer
// warps wait on "full", compute one block row each and arrive on "empty".
// No CTA-wide barrier: a warp that finishes its rows moves on to the next
// staged item.
template <int S>
__global__ void __launch_bounds__(STG_THREADS, 1) k_spmm_pipe(const PipeArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + MAX_STAGES;
    unsigned char* base = smem + 128;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            tc05::mbar_init(&full[s], PRODUCER_THREADS + 1);
            tc05::mbar_init(&empty[s], CONSUMER_WARPS);
        }
        tc05::fence_barrier_init();
    }
    __syncthreads();
    const int64_t G = gridDim.x;
    if (warp < PRODUCER_WARPS) {
        const int t = threadIdx.x;
        int64_t j = 0;
        for (int64_t item = blockIdx.x; item < a.n_items; item += G, ++j) {
            const int tile = (int)(item / a.nrt), r0 = (int)(item % a.nrt) * STG_KT;
            const int kt = min(STG_KT, a.k - r0);
            // this thread's column nodes, loaded before the stage wait so the loads overlap it
            const int c0 = a.tile_cptr[tile], nc = a.tile_cptr[tile + 1] - c0;
            int node[PRODUCER_PAIRS];
#pragma unroll
            for (int m = 0; m < PRODUCER_PAIRS; ++m) {
                const int e = t + m * PRODUCER_THREADS;
                node[m] = e < 2 * nc ? a.cols[c0 + (e >> 1)] : -1;
            }
            const int s = (int)(j % S);
            const uint32_t round = (uint32_t)(j / S);
            if (round > 0 && !bwait(&empty[s], (round - 1) & 1u)) {
                atomicOr(&g_staged_err, 1);
                break;
            }
            unsigned char* st = base + (size_t)s * a.stage_bytes;
            if (t == 0) {
                const int row0 = a.tile_row[tile], row1 = a.tile_row[tile + 1];
                const int blk0 = a.rp[row0], blk1 = a.rp[row1];
                const int mo0 = a.meta_off[tile], mo1 = a.meta_off[tile + 1];
                const uint32_t mbytes = (uint32_t)(blk1 - blk0) * 128u, tbytes = (uint32_t)(mo1 - mo0) * 16u;
                tc05::mbar_expect_tx(&full[s], mbytes + tbytes);
                tc05::bulk_g2s(st, a.val + 8 * (int64_t)blk0, mbytes, &full[s]);
                tc05::bulk_g2s(st + a.off_meta, a.meta + 16 * (int64_t)mo0, tbytes, &full[s]);
            }
            unsigned char* xs = st + a.off_x;
            const float2* xr = a.x + (int64_t)r0 * a.ldx;
#pragma unroll
            for (int m = 0; m < PRODUCER_PAIRS; ++m) {
                if (node[m] < 0) continue;
                const int e = t + m * PRODUCER_THREADS, cl = e >> 1, h = e & 1;
                const float2* src = xr + 4 * (int64_t)node[m] + 2 * h;
                unsigned char* dst = xs + (uint32_t)cl * 32u + (uint32_t)h * 16u;
                for (int q = 0; q < kt; ++q) cp_async16(dst + (uint32_t)q * a.xq, src + (int64_t)q * a.ldx);
            }
            cp_async_arrive_noinc(&full[s]);  // arrives once this thread's copies have landed
        }
        cp_async_wait<0>();
        return;
    }
    // ---- consumers: a warp takes 2 block rows at a time, 16 lanes per row, the two
    // half-warps on alternate blocks of the row; lane (pp, qq) of a row computes
    // the scalar row pair (2pp, 2pp + 1) for right-hand sides 2qq, 2qq + 1.  The
    // blocks are staged in the row-pair layout, so one 16-byte load holds column
    // c of both rows, (re, re, im, im): paired FMAs (fma.rn.f32x2) take the two
    // rows at once against the broadcast x entry, with the products of the
    // imaginary parts summed apart and subtracted at the end.  The half-warps'
    // partial sums meet in one shuffle.
    const int cw = warp - PRODUCER_WARPS, hh = lane >> 4, g = (lane >> 3) & 1, pp = (lane >> 2) & 1, qq = lane & 3;
    const int p0 = 2 * pp, q0 = 2 * qq;
    int64_t j = 0;
    for (int64_t item = blockIdx.x; item < a.n_items; item += G, ++j) {
        const int s = (int)(j % S);
        if (!bwait(&full[s], (uint32_t)(j / S) & 1u)) {
            if (lane == 0) atomicOr(&g_staged_err, 1);
            return;
        }
        const unsigned char* st = base + (size_t)s * a.stage_bytes;
        const int r0 = (int)(item % a.nrt) * STG_KT;
        const int kt = min(STG_KT, a.k - r0);
        const bool st0 = q0 < kt && (!a.active || a.active[r0 + q0]);
        const bool st1 = q0 + 1 < kt && (!a.active || a.active[r0 + q0 + 1]);
        const int32_t* hdr = reinterpret_cast<const int32_t*>(st + a.off_meta);
        const int row0 = hdr[0], row1 = hdr[1];  // from the staged metadata record
        const int32_t* rps = hdr + 4;
        const uint16_t* lcs = reinterpret_cast<const uint16_t*>(rps + (row1 - row0 + 1));
        const unsigned char* mb = st + (uint32_t)pp * 64u;
        const unsigned char* x0 = st + a.off_x + (uint32_t)q0 * a.xq;
        const unsigned char* x1 = x0 + a.xq;
        for (int i2 = row0 + 2 * cw; i2 < row1; i2 += 2 * CONSUMER_WARPS) {
            const int i = i2 + g;
            const bool row_ok = i < row1;
            const int s0 = row_ok ? rps[i - row0] : 0, s1 = row_ok ? rps[i - row0 + 1] : 0;
            const int64_t e0 = (int64_t)(r0 + q0) * a.ldy + 4 * (int64_t)i + p0;
            const int64_t e1 = e0 + a.ldy;
            float4 b0 = make_float4(0.f, 0.f, 0.f, 0.f), b1 = b0;  // in flight during the row
            if (a.b && row_ok && st0) b0 = *reinterpret_cast<const float4*>(a.b + e0);
            if (a.b && row_ok && st1) b1 = *reinterpret_cast<const float4*>(a.b + e1);
            // per right-hand side u (q0) and v (q0 + 1), each over the row pair:
            // sum re(m) re(x), sum im(m) im(x), sum of the imaginary part
            unsigned long long rpu = 0ull, rnu = 0ull, imu = 0ull, rpv = 0ull, rnv = 0ull, imv = 0ull;
            for (int sb = s0 + hh; sb < s1; sb += 2) {  // the two half-warps take alternate blocks
                const uint32_t lc = lcs[sb];
                const ulonglong2* m = reinterpret_cast<const ulonglong2*>(mb + (uint32_t)sb * 128u);
                const float4* u = reinterpret_cast<const float4*>(x0 + lc * 32u);
                const float4* v = reinterpret_cast<const float4*>(x1 + lc * 32u);
                const float4 ua = u[0], ub = u[1], va = v[0], vb = v[1];
                const float xu[8] = {ua.x, ua.y, ua.z, ua.w, ub.x, ub.y, ub.z, ub.w};
                const float xv[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    const ulonglong2 mc = m[cc];  // (re row p0, re row p0 + 1), (im, im) of column cc
                    const unsigned long long ur = f2pack(xu[2 * cc], xu[2 * cc]), ui = f2pack(xu[2 * cc + 1], xu[2 * cc + 1]);
                    const unsigned long long vr = f2pack(xv[2 * cc], xv[2 * cc]), vi = f2pack(xv[2 * cc + 1], xv[2 * cc + 1]);
                    rpu = ffma2(mc.x, ur, rpu);
                    rnu = ffma2(mc.y, ui, rnu);
                    imu = ffma2(mc.x, ui, imu);
                    imu = ffma2(mc.y, ur, imu);
                    rpv = ffma2(mc.x, vr, rpv);
                    rnv = ffma2(mc.y, vi, rnv);
                    imv = ffma2(mc.x, vi, imv);
                    imv = ffma2(mc.y, vr, imv);
                }
            }
            float o[8];  // (re, im) of rows p0, p0 + 1 for u, then for v
            {
                float a0, a1, n0, n1, i0, i1;
                f2unpack(rpu, a0, a1);
                f2unpack(rnu, n0, n1);
                f2unpack(imu, i0, i1);
                o[0] = a0 - n0, o[1] = i0, o[2] = a1 - n1, o[3] = i1;
                f2unpack(rpv, a0, a1);
                f2unpack(rnv, n0, n1);
                f2unpack(imv, i0, i1);
                o[4] = a0 - n0, o[5] = i0, o[6] = a1 - n1, o[7] = i1;
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) o[e] += __shfl_xor_sync(0xffffffffu, o[e], 16);  // the other half-warp
            if (!row_ok || hh) continue;
            if (st0) {
                float4 r = make_float4(o[0], o[1], o[2], o[3]);
                if (a.b) r = make_float4(b0.x - r.x, b0.y - r.y, b0.z - r.z, b0.w - r.w);
                *reinterpret_cast<float4*>(a.y + e0) = r;
            }
            if (st1) {
                float4 r = make_float4(o[4], o[5], o[6], o[7]);
                if (a.b) r = make_float4(b1.x - r.x, b1.y - r.y, b1.z - r.z, b1.w - r.w);
                *reinterpret_cast<float4*>(a.y + e1) = r;
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
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
        // shorten the tile until its column list fits the producers and the plan's stage
        // (the largest blocks, metadata and list over its tiles) still fits twice in shared
        // memory (rows with many blocks spread over many columns, as on coarse levels)
        auto meta_bytes = [&](int64_t e_) {
            return (int)((16 + (size_t)(e_ - i + 1) * 4 + (size_t)(rp[e_] - rp[i]) * 2 + 15) / 16 * 16);
        };
        auto fits = [&](int64_t e_, int nc_) {
            if (nc_ > MAX_TILE_COLS) return false;
            const StageLayout L = stage_layout(std::max<int>(P.max_blocks, rp[e_] - rp[i]),
                                               std::max<int>(P.max_meta, meta_bytes(e_)), std::max<int>(P.max_cols, nc_));
            return L.stages >= 2;
        };
        int nc = cover(col, rp[i], rp[e], cols, list);
        while (!fits(e, nc) && e > i + 1) {
            --e;
            nc = cover(col, rp[i], rp[e], cols, list);
        }
        if (!fits(e, nc)) return;
        blocks = rp[e] - rp[i];
        for (int u = 0; u < nc; ++u) loc[list[u]] = u;
        // metadata record: first and end row (int32, then 2 pad words), row offsets (int32),
        // local columns (uint16), padded to 16 bytes
        const size_t m0 = meta.size();
        const int64_t nr = e - i;
        const size_t bytes = 16 + (size_t)(nr + 1) * 4 + (size_t)blocks * 2;
        meta.resize(m0 + (bytes + 15) / 16 * 16, 0);
        int32_t* hd = reinterpret_cast<int32_t*>(meta.data() + m0);
        hd[0] = (int32_t)i;
        hd[1] = (int32_t)e;
        int32_t* ro = hd + 4;
        uint16_t* lc = reinterpret_cast<uint16_t*>(meta.data() + m0 + 16 + (size_t)(nr + 1) * 4);
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

// row-pair layout: block b, float4 4P + c = (re A[2P][c], re A[2P+1][c], im A[2P][c], im A[2P+1][c])
__global__ void k_to_pair(const float2* __restrict__ in, float4* __restrict__ out, int64_t nnzb) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // (block, P, c)
    if (e >= 8 * nnzb) return;
    const int64_t b = e >> 3;
    const int P = (int)(e >> 2) & 1, c = (int)e & 3;
    const float2 lo = in[16 * b + 4 * (2 * P) + c], hi = in[16 * b + 4 * (2 * P + 1) + c];
    out[e] = make_float4(lo.x, hi.x, lo.y, hi.y);
}

__global__ void k_to_transposed(const float2* __restrict__ in, float2* __restrict__ out, int64_t nnzb) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // (block, row p, column r)
    if (e >= 16 * nnzb) return;
    const int64_t b = e >> 4;
    const int p = (int)(e >> 2) & 3, r = (int)e & 3;
    out[16 * b + 4 * r + p] = in[e];
}

void to_pair_layout(cudaStream_t st, const float2* in, float4* out, int64_t nnzb) {
    if (nnzb <= 0) return;
    k_to_pair<<<grid_for(8 * nnzb, 256), 256, 0, st>>>(in, out, nnzb);
    ECT_CHECK_LAUNCH();
}

void to_transposed_layout(cudaStream_t st, const float2* in, float2* out, int64_t nnzb) {
    if (nnzb <= 0) return;
    k_to_transposed<<<grid_for(16 * nnzb, 256), 256, 0, st>>>(in, out, nnzb);
    ECT_CHECK_LAUNCH();
}

void bsr_spmm_staged_f32(cudaStream_t st, const StagedPlan& P, const int32_t* rp, const float4* val,
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
