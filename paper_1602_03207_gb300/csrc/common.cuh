// Shared device helpers and the library context of the eddy-current solver.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <cmath>
#include <cstring>
#include <deque>
#include <functional>
#include <string>
#include <vector>

#include "../../include/ect.h"

// ----------------------------------------------------------------------------
// complex arithmetic on double2 / float2 (x = re, y = im)
// ----------------------------------------------------------------------------
template <typename T> struct cplx;
template <> struct cplx<double> { using type = double2; };
template <> struct cplx<float> { using type = float2; };
template <typename T> using C = typename cplx<T>::type;

__host__ __device__ __forceinline__ double2 mk(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ float2 mk(float r, float i) { return make_float2(r, i); }
template <typename T> __host__ __device__ __forceinline__ C<T> czero() { return mk(T(0), T(0)); }

// acc += a * b
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cfma_conj(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma_conj(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(-a.y, b.x, acc.y);
}
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

__device__ __forceinline__ double2 to_d(float2 a) { return make_double2(a.x, a.y); }
__device__ __forceinline__ double2 to_d(double2 a) { return a; }
template <typename T> __device__ __forceinline__ C<T> from_d(double2 a);
template <> __device__ __forceinline__ double2 from_d<double>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from_d<float>(double2 a) { return make_float2((float)a.x, (float)a.y); }

// warp sum of a double
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ----------------------------------------------------------------------------
// error handling
// ----------------------------------------------------------------------------
struct EctError {
    int code;
    std::string msg;
};

#define ECT_CUDA(call)                                                                        \
    do {                                                                                      \
        cudaError_t _e = (call);                                                              \
        if (_e != cudaSuccess) {                                                              \
            throw EctError{_e == cudaErrorMemoryAllocation ? ECT_ERR_OOM : ECT_ERR_CUDA,       \
                           std::string(#call) + ": " + cudaGetErrorString(_e)};               \
        }                                                                                     \
    } while (0)

#define ECT_CHECK_LAUNCH() ECT_CUDA(cudaGetLastError())

#define ECT_REQUIRE(cond, code, msg)                  \
    do {                                              \
        if (!(cond)) throw EctError{(code), (msg)};   \
    } while (0)

inline unsigned grid_for(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    return (unsigned)g;
}

// The FP32 block inverses are stored packed: the inverse of a complex
// symmetric block is complex symmetric, so only its upper triangle is kept,
// column by column (entry (i, j), i <= j, at j (j + 1) / 2 + i).  b = 4 n is
// a multiple of 4, so every packed block has an even length and every block
// starts 16-byte aligned.
inline int64_t sym_packed_size(int b) { return (int64_t)b * (b + 1) / 2; }

// one-dimensional grid of row_blocks x n_tiles CTAs (tile index fastest)
inline unsigned tile_grid(unsigned row_blocks, int n_tiles) {
    const int64_t g = (int64_t)row_blocks * n_tiles;
    if (g > 0x7fffffffLL) throw EctError{ECT_ERR_ARG, "launch grid too large"};
    return (unsigned)g;
}

// right-hand-side tile of the multi-RHS kernels: the requested size (0: 8)
// rounded down to a power of two <= 8 and <= k
inline int pick_tile(int k, int rhs_tile) {
    int kt = rhs_tile > 0 ? rhs_tile : 8;
    if (kt > k) kt = k;
    if (kt >= 8) return 8;
    if (kt >= 4) return 4;
    if (kt >= 2) return 2;
    return 1;
}

// Cover k right-hand sides with full tiles: as many of the preferred tile as
// fit, then smaller powers of two for the rest.  launch(kt, first_rhs, n_tiles)
// is called once per tile size.
template <typename L>
void for_tiles(int k, int rhs_tile, L launch) {
    for (int done = 0; done < k;) {
        const int kt = pick_tile(k - done, rhs_tile);
        const int nt = (k - done) / kt;
        launch(kt, done, nt);
        done += nt * kt;
    }
}

// ----------------------------------------------------------------------------
// device buffer
// ----------------------------------------------------------------------------
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    void alloc(size_t nbytes) {
        if (nbytes == bytes && p) return;
        release();
        if (nbytes == 0) return;
        ECT_CUDA(cudaMalloc(&p, nbytes));
        bytes = nbytes;
    }
    void ensure(size_t nbytes) {
        if (nbytes > bytes) alloc(nbytes);
    }
    template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

// ----------------------------------------------------------------------------
// staged FP32 SpMM (spmm_staged.cu): a BSR matrix cut into tiles of
// consecutive block rows; each tile lists the distinct column nodes its
// blocks touch, and every block stores its column as an index into that list
// ----------------------------------------------------------------------------
struct StagedPlan {
    bool ok = false;       // false: some row alone exceeds the tile limits (use the unstaged kernels)
    int rows = 0;          // target block rows per tile
    int64_t n_rows = 0, n_tiles = 0;
    int max_cols = 0, max_blocks = 0;  // over all tiles (they size the shared memory)
    int max_meta = 0;      // bytes of the largest tile's metadata record
    DevBuf tile_row;       // int32[n_tiles+1] first block row of each tile
    DevBuf tile_cptr;      // int32[n_tiles+1] offsets into the tiles' column lists
    DevBuf tile_meta_off;  // int32[n_tiles+1] offsets (16-byte units) of each tile's metadata record
    DevBuf tile_meta;      // per tile: row offsets (int32, rows+1) and local column indices
                           // (uint16 per block), padded to 16 bytes
    DevBuf tile_cols;      // int32 column nodes of each tile's list (runs of consecutive nodes)
    void reset() {
        ok = false;
        rows = 0;
        n_rows = n_tiles = 0;
        max_cols = max_blocks = max_meta = 0;
        for (DevBuf* b : {&tile_row, &tile_cptr, &tile_meta_off, &tile_meta, &tile_cols}) b->release();
    }
};
// Build the plan of a BSR pattern (host arrays) for tiles of about `rows`
// block rows; columns index a space of n_cols nodes.
void staged_plan_build(cudaStream_t st, StagedPlan& P, const std::vector<int32_t>& rp,
                       const std::vector<int32_t>& col, int64_t n_rows, int64_t n_cols, int rows);
// y[r] = A x[r] (b == nullptr) or y[r] = b[r] - A x[r] for k right-hand sides
// (b may equal y: in-place t -= A x).  x has leading dimension ldx (column
// space), b and y ldy (row space).  FP32 complex values in the row-pair
// layout (to_pair_layout), 8 float4 per block.
void bsr_spmm_staged_f32(cudaStream_t st, const StagedPlan& P, const int32_t* rp, const float4* val,
                         const float2* x, int64_t ldx, const float2* b, float2* y, int64_t ldy, int k,
                         const int* active);
// Block layouts of FP32 4x4 complex blocks stored row-major (16 float2 per block):
// the row-pair layout of the staged SpMM and the transposed layout of the
// warp-per-row SpMM.
void to_pair_layout(cudaStream_t st, const float2* in, float4* out, int64_t nnzb);
void to_transposed_layout(cudaStream_t st, const float2* in, float2* out, int64_t nnzb);
// Read and clear the flag that a staged kernel sets when its bounded wait on
// a bulk copy expired (1 = expired).  Synchronises the stream.
int staged_take_error(cudaStream_t st);
// FP32 SpMM with one warp per block row: lane (p, q) takes column p of every
// block (from the transposed copy) and right-hand side q, and the four
// partial rows are summed with shuffles at the end of the row (spmv.cu)
void bsr_spmm_colwarp_f32(cudaStream_t st, const int32_t* rp, const int32_t* col, const float2* valt, int64_t N,
                          const float2* x, int64_t ldx, const float2* b, float2* y, int64_t ldy, int k,
                          const int* active);
constexpr int SPMM_COLWARP = -2;  // ect_options.spmm_rows value selecting it

// Paired single-precision FMA (two lanes of a 64-bit register pair per
// instruction, sm_100 family): d = a * b + c elementwise.
__device__ __forceinline__ unsigned long long f2pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2unpack(unsigned long long v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// default target rows per tile of the staged SpMM
constexpr int STAGED_ROWS_DEFAULT = 32;

// ----------------------------------------------------------------------------
// context
// ----------------------------------------------------------------------------
struct Multigrid;  // aggregation multigrid hierarchy (multigrid.cu)
struct Matrix;
void mg_free(Matrix& M);

struct Matrix {
    double omega = 0.0;    // angular frequency of the assembled values
    bool assembled = false;
    bool has_f32 = false;
    bool pc_f64 = false, pc_f32 = false;
    DevBuf sigma, nu;      // per tet, effective coefficients of this configuration
    DevBuf fixmask;        // uint8 per node: bits 0-2 Dirichlet A, bit 3 V identity
    DevBuf val;            // double2[nnzb*16] unscaled, constrained
    DevBuf sval;           // double2[nnzb*16] scaled  S = T M T
    DevBuf sval32;         // float2 [nnzb*16] scaled
    DevBuf sval32lo;       // float2 [nnzb*16] FP32 remainder: sval ~= sval32 + sval32lo to ~2^-48
    DevBuf sval32p;        // float4 [nnzb*8] FP32 scaled, row-pair layout (the staged SpMM's input):
                           //   per block, rows (2P, 2P+1) and column c at float4 4P + c:
                           //   (re S[2P][c], re S[2P+1][c], im S[2P][c], im S[2P+1][c])
    DevBuf sval32t;        // float2 [nnzb*16] FP32 scaled, each block transposed (column-major);
                           //   built from sval32 when the warp-per-row SpMM is selected
    uint64_t val_gen = 0;  // bumped whenever the scaled values are rewritten
    uint64_t t_gen = 0;    // val_gen that sval32t was built from (0: never)
    DevBuf t;              // double[4N] scaling
    DevBuf pinv;           // double2 block inverses (column-major per block)
    DevBuf pinv32;         // float2  block inverses
    // conductor-V coarse space (two-level preconditioner)
    int64_t nc = 0;        // coarse unknowns (0 = one-level)
    int coarse_group = 0;
    DevBuf einv, einv32;   // E^-1 (nc x nc, symmetric), FP64 and FP32
    DevBuf blk_c;          // int32[n_blocks] coarse index of each subdomain, -1 if none
    DevBuf agg_lo, agg_hi; // int32[nc] node range of each coarse group
    DevBuf zv, zv32;       // 1/t at the V dof of conducting nodes, 0 elsewhere (N)
    DevBuf rc, zc;         // coarse scratch [k][nc] (double2 or float2 storage)
    DevBuf gpart;          // split-GEMV partial sums
    int64_t coarse_k = 0;
    std::vector<uint8_t> h_cond;  // conducting-node flags (host)
    std::vector<uint8_t> h_fix;   // host copy of fixmask
    std::vector<double> h_sigma, h_nu;  // per-tet coefficients of this configuration (host)
    // impedance boundary condition (Eq. IBC): plate tets removed, surface term on their boundary
    int pc_mask = 0, pc_group = 0;  // arguments of the last ect_precond_setup
    bool ibc = false;
    double ibc_sigma = 0.0, ibc_nu = 0.0;  // plate conductivity and 1/mu
    std::vector<uint8_t> h_void;  // per tet: 1 = plate (removed from the volume forms)
    DevBuf tvoid;          // uint8[T]
    DevBuf s_ptr;          // int32[nnzb+1] per block: range of its surface contributions
    DevBuf s_ent;          // uint32 face<<4 | a<<2 | b
    DevBuf s_geo;          // double[F][4]: area, unit normal into the plate
    int64_t n_faces = 0;
    Multigrid* mg = nullptr;
    Matrix() = default;
    Matrix(const Matrix&) = delete;
    Matrix& operator=(const Matrix&) = delete;
    ~Matrix() { mg_free(*this); }
    void reset() {
        mg_free(*this);
        assembled = has_f32 = pc_f64 = pc_f32 = false;
        nc = 0;
        coarse_group = 0;
        coarse_k = 0;
        h_cond.clear();
        h_fix.clear();
        ibc = false;
        h_void.clear();
        n_faces = 0;
        for (DevBuf* b : {&tvoid, &s_ptr, &s_ent, &s_geo}) b->release();
        for (DevBuf* b : {&sigma, &nu, &fixmask, &val, &sval, &sval32, &sval32lo, &sval32p, &sval32t, &t, &pinv, &pinv32, &einv, &einv32, &blk_c,
                          &agg_lo, &agg_hi, &zv, &zv32, &rc, &zc, &gpart})
            b->release();
    }
};

struct Workspace;  // Krylov workspace (krylov.cu)

struct ect_ctx {
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;
    // physics
    double freq = 1.0e5, omega = 2.0 * 3.14159265358979323846 * 1.0e5;
    double nu_tilde = 0.0, delta = 1.0;
    bool physics_set = false;
    // mesh
    bool mesh_set = false;
    int64_t n_nodes = 0, n_tets = 0, nnzb = 0, n_blocks = 0, n_entries = 0;
    int max_block_nodes = 0;
    DevBuf xyz;            // double[N*3]
    DevBuf tets;           // int32[T*4]
    DevBuf geo;            // double[T*16]: vol, g0..g3 (xyz), pad
    DevBuf bc;             // uint8[N]
    DevBuf row_ptr;        // int32[N+1]
    DevBuf col;            // int32[nnzb]
    DevBuf diag_slot;      // int32[N]
    DevBuf slot_ptr;       // int32[nnzb+1]
    DevBuf entries;        // uint32[16T]: tet<<4 | a<<2 | b
    DevBuf block_ptr;      // int32[n_blocks+1] node offsets
    DevBuf pinv_off;       // int64[n_blocks+1] offsets (in complex entries) of block inverses
    int64_t pinv_total = 0;
    DevBuf pinv_off32;     // int64[n_blocks+1] offsets of the packed FP32 (upper triangle) inverses
    int64_t pinv_total32 = 0;
    DevBuf omega_d;        // int32 list of defect tets
    int64_t n_omega_d = 0;
    std::vector<int32_t> h_block_ptr;       // smoothing blocks (the subdomains, possibly split)
    std::vector<int32_t> h_block_ptr_mesh;  // the subdomains given with the mesh
    int block_split = 1;                    // pieces per subdomain
    std::vector<int32_t> h_row_ptr, h_col;
    std::vector<int32_t> h_tets;
    std::vector<uint8_t> h_bc;
    std::vector<double> h_sigma0, h_nu0;
    Matrix mat[2];
    // frequency sweep: configuration c at sweep frequency f is smat[2 f + c] (which = 2 + 2 f + c)
    std::vector<double> sweep_omega;
    std::deque<Matrix> smat;
    StagedPlan fine_plan;  // staged-SpMM tiling of the (shared) finest pattern
    int staged_rows = STAGED_ROWS_DEFAULT;  // rows per staged tile of the FP32 SpMM; -1 = unstaged
    int kernel_rows = STAGED_ROWS_DEFAULT;  // staged tiling used by ect_spmv / ect_precond_apply
    int plan_gen = 0;      // bumped whenever a staged plan is rebuilt (captured graphs key on it)
    Workspace* ws = nullptr;
    // scratch
    DevBuf scratch;        // reduction partials etc.
    DevBuf pinned;         // host-visible small results
    void* h_pinned = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

// matrix `which`: 0 / 1 the two configurations at the context's frequency,
// 2 + 2 f + c configuration c at sweep frequency f
inline bool which_valid(const ect_ctx* c, int which) {
    return which == ECT_VACUUM || which == ECT_DEFECT || (which >= 2 && which < 2 + (int)c->smat.size());
}
inline Matrix& ctx_mat(ect_ctx* c, int which) {
    if (which == ECT_VACUUM || which == ECT_DEFECT) return c->mat[which];
    if (which >= 2 && which < 2 + (int)c->smat.size()) return c->smat[which - 2];
    throw EctError{ECT_ERR_ARG, "which must be ECT_VACUUM, ECT_DEFECT or a sweep matrix (ECT_SWEEP_MATRIX)"};
}
inline double ctx_omega(const ect_ctx* c, int which) {
    return which >= 2 ? c->sweep_omega[(which - 2) / 2] : c->omega;
}

// shared scratch (partials) helper
inline double* ctx_scratch(ect_ctx* c, size_t doubles) {
    c->scratch.ensure(doubles * sizeof(double));
    return c->scratch.as<double>();
}

// Run f and turn any exception into a status code and c->err (the message of
// the last error); implemented in api.cu, used by every extern "C" entry point.
int guarded_call(ect_ctx* c, const std::function<void()>& f);

// ----------------------------------------------------------------------------
// cross-file entry points (implemented in the .cu files)
// ----------------------------------------------------------------------------
void mesh_setup(ect_ctx* c, const double* xyz, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                const double* sigma, const double* nu, const double* sigma_d, const double* nu_d,
                const int32_t* block_of_node, const uint8_t* bc_mask);
void set_defect(ect_ctx* c, const double* sigma_d, const double* nu_d);
void set_ibc(ect_ctx* c, int which, const uint8_t* plate, double sigma_p, double nu_p);
// per-tet coefficients, conducting nodes and constraint mask of configuration m (mesh_setup.cu)
void upload_config(ect_ctx* c, int m, const std::vector<double>& s, const std::vector<double>& n);
// recursive coordinate bisection into contiguous subdomains of at most s nodes (partition.cu)
void partition_rcb(const double* xyz, int64_t n_nodes, int s, int32_t* new_id, int32_t* block_of_new);
void assemble_matrix(ect_ctx* c, int which, int precision_mask);
void precond_setup(ect_ctx* c, int which, int precision_mask, int coarse_group);
void coarse_scratch(ect_ctx* c, int which, int k);
void mg_setup(ect_ctx* c, int which, bool f32);
void mg_scratch(Matrix& M, int k);
// (re)build the staged-SpMM plans of the finest pattern and of the multigrid
// levels of `which` for c->staged_rows (no-op when they match); not capturable
void staged_prepare(ect_ctx* c, int which);
void mg_apply_f64(ect_ctx* c, int which, const double2* r, double2* z, int k, int64_t ld, int tile, const int* active);
void mg_apply_f32(ect_ctx* c, int which, const float2* r, float2* z, int k, int64_t ld, int tile, const int* active);
int mg_levels(const Matrix& M);
bool mg_ready(const Matrix& M, int k);

// y = A x for k vectors; A = unscaled F64 (scaled=false) or scaled S (scaled=true)
void spmv_f64(ect_ctx* c, int which, bool scaled, const double2* x, double2* y, int k, int64_t ldx,
              int rhs_tile, const int* active);
void spmv_f32(ect_ctx* c, int which, const float2* x, float2* y, int k, int64_t ldx, int rhs_tile,
              const int* active);
// y (FP64) = S u for u exactly representable in FP32 (double-float arithmetic
// on sval32 + sval32lo); used by the mixed mode's outer Arnoldi step
void spmv_df32(ect_ctx* c, int which, const float2* u, double2* y, int k, int64_t ldx, int rhs_tile,
               const int* active);
void precond_apply_f64(ect_ctx* c, int which, const double2* r, double2* z, int k, int64_t ld,
                       int rhs_tile, const int* active);
void precond_apply_f32(ect_ctx* c, int which, const float2* r, float2* z, int k, int64_t ld,
                       int rhs_tile, const int* active);
// generic building blocks (spmv.cu, precond.cu) shared by the multigrid levels
void bsr_spmv_f64(cudaStream_t st, const int32_t* rp, const int32_t* cl, const double2* val, int64_t N,
                  const double2* x, const double2* b, double2* y, int k, int64_t ldx, int rhs_tile, const int* active);
void bsr_spmv_f32(cudaStream_t st, const int32_t* rp, const int32_t* cl, const float2* val, int64_t N,
                  const float2* x, const float2* b, float2* y, int k, int64_t ldx, int rhs_tile, const int* active);
// one warp per block row (coarse multigrid levels: few rows, many blocks per row)
template <typename T>
void bsr_spmv_warp(cudaStream_t st, const int32_t* rp, const int32_t* cl, const C<T>* val, int64_t N, const C<T>* x,
                   const C<T>* b, C<T>* y, int k, int64_t ldx, int rhs_tile, const int* active);
void block_inverses(cudaStream_t st, const int32_t* rp, const int32_t* col, const double2* sval, const int32_t* bptr,
                    const int64_t* poff, const int64_t* poff32, int64_t n_blocks, int max_block_nodes, double2* pinv,
                    float2* pinv32);
// z = S_ss^-1 r per smoothing block (accumulate: z += ...); for T = float, pinv
// and poff are the packed FP32 inverses and their offsets
template <typename T>
void block_apply(cudaStream_t st, const int32_t* bptr, const int64_t* poff, const C<T>* pinv, int64_t n_blocks,
                 int max_block_nodes, const C<T>* r, C<T>* z, int k, int64_t ld, int rhs_tile, const int* active,
                 bool accumulate);
void dense_inverse(cudaStream_t st, double2* a, int64_t n);
void to_f32(cudaStream_t st, const double2* a, float2* b, int64_t n);
int64_t gemv_scratch_elems(int64_t nc, int k);
template <typename T>
void dense_gemv(cudaStream_t st, const C<T>* einv, int64_t nc, const C<T>* r, C<T>* z, int k, int rhs_tile,
                const int* active, C<T>* part);

void coil_rhs(ect_ctx* c, const ect_coil& coil, const double* h_z, int k, double2* d_rhs);
// omega: the angular frequency of the solutions (0: the context's)
void delta_z(ect_ctx* c, const double2* u0, const double2* ud, const double2* b, const double* cur,
             int n_pos, double* h_dz, double* h_dz_emf, double omega = 0.0);
// drop the frequency-sweep matrices (their coefficients changed)
void clear_sweep(ect_ctx* c);
// smoothing blocks from the mesh's subdomains and c->block_split (mesh_setup.cu)
void apply_block_split(ect_ctx* c);
// cut every subdomain into `parts` pieces; every preconditioner must be set up again
void set_block_split(ect_ctx* c, int parts);
void solve(ect_ctx* c, int which, const double2* rhs, double2* x, int k, const ect_options& opt,
           ect_stats* st);
// all sweep frequencies of configuration `config` in one lockstep solve: rhs, x [F][k][4N]
// (same_rhs: one rhs array [k][4N] serves every frequency)
void solve_sweep(ect_ctx* c, int config, const double2* rhs, double2* x, int k, const ect_options& opt,
                 ect_stats* st, bool same_rhs = false);
void assemble_sweep(ect_ctx* c, const double* freq_hz, int n_freq, int precision_mask);
void cgs2_entry(ect_ctx* c, int precision, const void* V, int j, int64_t n, void* w, double* h,
                double* beta);
void workspace_free(ect_ctx* c);
