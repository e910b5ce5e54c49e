/*
 * ect.h - C ABI of the GB300 eddy-current finite-element solver.
 *
 * The library assembles and solves the discrete time-harmonic eddy-current
 * problem in the Coulomb-gauged A-V potential formulation with P1 nodal
 * elements on tetrahedra (Riahi, "A Fast Eddy-current Non Destructive Testing
 * Finite Element Solver in Steam Generator", Sec. 2-3), and reads out the
 * coil-impedance change Delta Z of Eq. impedkl for each probe position.
 *
 * Conventions for every entry point
 *   - Return value: ECT_OK (0) or one of the ECT_ERR_* codes below; on error
 *     ect_last_error() describes it.  No C++ exception crosses the ABI.
 *   - Pointers prefixed h_ are host memory, d_ device memory (any allocator,
 *     e.g. torch tensors).  Host inputs are copied; the caller keeps
 *     ownership of every buffer it passes.
 *   - Complex values are interleaved (re, im) pairs: double[2] for complex128,
 *     float[2] for complex64.
 *   - Unknowns are ordered per node as (A_x, A_y, A_z, V); a vector of one
 *     right-hand side has 4*n_nodes complex entries, dof = 4*node + comp.
 *     A batch of k vectors is stored [k][n_nodes][4] (each vector contiguous).
 *   - All GPU work is enqueued on the stream given to ect_create; calls that
 *     return host data synchronise that stream.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef ECT_H
#define ECT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------- */
#define ECT_OK 0
#define ECT_ERR_ARG 1            /* invalid argument (null, size, range)       */
#define ECT_ERR_MESH 2           /* bad mesh: index out of range, volume <= 0  */
#define ECT_ERR_CUDA 3           /* a CUDA call failed                          */
#define ECT_ERR_OOM 4            /* device allocation failed                    */
#define ECT_ERR_NOT_CONVERGED 5  /* tolerance not met; x and stats are filled   */
#define ECT_ERR_BREAKDOWN 6      /* NaN/Inf in the Krylov recurrence            */
#define ECT_ERR_TIMEOUT 7        /* options.timeout_s expired; x is filled      */
#define ECT_ERR_STATE 8          /* call out of order (e.g. solve before assemble) */

/* ---- which matrix ---------------------------------------------------------- */
#define ECT_VACUUM 0             /* background configuration ("vacuum", Sec. 2 remark) */
#define ECT_DEFECT 1             /* configuration with the defect region Omega_d       */

/* ---- precision ------------------------------------------------------------- */
#define ECT_F64 1                /* complex128 */
#define ECT_F32 2                /* complex64  */

/* solver modes (ect_options.mode) */
#define ECT_MODE_F64 0           /* flexible GMRES, everything in FP64                   */
#define ECT_MODE_MIXED 1         /* FP64 flexible GMRES outer loop, FP32 GMRES inner solve */

typedef struct ect_ctx ect_ctx;

/* Annular coil with azimuthal current density J_e (Sec. 4): it occupies
 * r_in <= r <= r_out around the z axis and |z - (z_probe + z_offset)| <= length/2.
 * Lengths in metres, J_e in A/m^2. */
typedef struct {
    double r_in, r_out, length, z_offset, J_e;
} ect_coil;

typedef struct {
    double tol;         /* relative residual ||T(b - M x)|| / ||T b|| (T = diag |M_ii|^-1/2) */
    int restart;        /* Krylov restart length m (outer length in mixed mode)           */
    int max_iters;      /* cap on outer iterations (F64: all iterations)                  */
    int mode;           /* ECT_MODE_F64 or ECT_MODE_MIXED                                 */
    int inner_iters;    /* mixed mode: FP32 GMRES iterations per outer step               */
    int use_graph;      /* 1: replay each restart cycle as a captured CUDA graph           */
    int rhs_tile;       /* right-hand sides per SpMM/preconditioner pass (0 = auto, 8);
                           -1 = FP32 SpMM variant that splits the tile over thread groups */
    double timeout_s;   /* wall-clock limit of one solve call (0 = none)                  */
    int reorth;         /* 0: always two Gram-Schmidt passes; 1: second pass only when the
                           first removed more than half of ||w||^2 (default); 2: as 1 in
                           the FP64 loop, one classical pass in the mixed mode's FP32 loop;
                           3: one classical pass in both loops                           */
    int spmm_rows;      /* FP32 SpMM variant: > 0 block rows per shared-memory-staged tile;
                           0 = auto (32); -1 = one thread per scalar row (x gathered from
                           L1/L2); -2 = one warp per block row over the transposed blocks */
    int x0;             /* ect_solve / ect_solve_sweep: 1 = d_x holds an initial guess (for
                           example the background solution when solving the defect
                           configuration), 0 = start from zero (d_x need not be initialised).
                           The tolerance stays relative to ||T b||.  Ignored by the calls that
                           own their solution buffers (impedance, autotune). */
} ect_options;

typedef struct {
    int iters;          /* Krylov iterations (inner ones in mixed mode), max over rhs */
    int outer_iters;    /* outer iterations, max over rhs                             */
    int converged;      /* number of right-hand sides that met tol                    */
    int restarts;       /* restart cycles run                                          */
    double relres_max;  /* max over rhs of the true relative residual at exit          */
    double ms;          /* device time of the call (CUDA events on the context stream) */
    int64_t launches;   /* kernels launched (graph nodes x replays + direct launches); counted
                           for the graph path, 0 when graphs are off                      */
} ect_stats;

/* Fill *opt with defaults: tol 1e-10, restart 30, max_iters 20000, F64 mode,
 * inner_iters 30, graphs on, automatic rhs tile, no timeout, selective
 * reorthogonalisation, staged FP32 SpMM with automatic row tiling, zero
 * initial guess. */
void ect_default_options(ect_options* opt);

/* Create a context bound to a CUDA stream (a cudaStream_t, may be NULL for the
 * legacy default stream) on the current device.  Free with ect_destroy. */
int ect_create(ect_ctx** out, void* cuda_stream);
void ect_destroy(ect_ctx* ctx);

/* Message of the last error on this context (or of the last failed
 * ect_create on this thread when ctx is NULL).  Never NULL. */
const char* ect_last_error(const ect_ctx* ctx);

/* Step 1-2 of Sec. 3: the triangulation and its partition.
 *   h_xyz            double[n_nodes][3] node coordinates (metres)
 *   h_tets           int32[n_tets][4] node indices, positively oriented
 *   h_sigma, h_nu    double[n_tets] background conductivity and 1/mu
 *   h_sigma_d, h_nu_d double[n_tets] defect configuration; NaN = same as background
 *                    (both may be NULL: no defect)
 *   h_block_of_node  int32[n_nodes] subdomain id of each node; must be
 *                    non-decreasing from 0 in steps of 0 or 1 (each subdomain a
 *                    contiguous node range of at most 16 nodes)
 *   h_bc_mask        uint8[n_nodes] bit c set = A component c (0=x,1=y,2=z) is
 *                    fixed to 0 at that node (A.n = 0 on the box faces, Sec. 3)
 * Builds the block-sparse pattern on the device.  ECT_ERR_MESH on an index
 * out of range or a tet of non-positive volume. */
int ect_set_mesh(ect_ctx* ctx, const double* h_xyz, int64_t n_nodes,
                 const int32_t* h_tets, int64_t n_tets,
                 const double* h_sigma, const double* h_nu,
                 const double* h_sigma_d, const double* h_nu_d,
                 const int32_t* h_block_of_node, const uint8_t* h_bc_mask);

/* Step 2 of Sec. 3 for meshes that come without a partition (e.g. from a
 * mesh generator): recursive coordinate bisection of the nodes into
 * subdomains of at most max_block_nodes (1..16) nodes.
 *   h_xyz           double[n_nodes][3] node coordinates
 *   h_new_id        int32[n_nodes] out: new index of node i
 *   h_block_of_new  int32[n_nodes] out: subdomain of new node j, non-decreasing
 *                   from 0 in steps of 0 or 1 (the order ect_set_mesh needs)
 * Relabel the mesh with h_new_id (tets, coordinates, per-node arrays) before
 * ect_set_mesh.  Host-only, deterministic, needs no context (errors:
 * ect_last_error(NULL)). */
int ect_partition(const double* h_xyz, int64_t n_nodes, int max_block_nodes, int32_t* h_new_id,
                  int32_t* h_block_of_new);

/* Replace the defect configuration (h_sigma_d, h_nu_d as in ect_set_mesh;
 * NaN = background, NULL = no defect) on the current mesh without rebuilding
 * the pattern: the defect matrix and its preconditioner must be assembled
 * and set up again.  Used to scan many deposits on one mesh. */
int ect_set_defect(ect_ctx* ctx, const double* h_sigma_d, const double* h_nu_d);

/* Impedance boundary condition (Sec. 2, Eq. IBC with the surface integral of
 * Eq. ibcROTA) for configuration `which`: the tets with h_tet_plate[t] != 0
 * (a good conductor, e.g. the support plate, of conductivity sigma_p and
 * reluctivity nu_p = 1/mu_p) are removed from the volume forms, every dof of
 * a node that touches only plate tets is fixed to zero, and on the plate's
 * surface (faces shared with the remaining tets, normal n into the plate)
 * the A-A block receives -(i omega / Z) int A_tau . Phi_tau with
 * Z = (1 - i)/(delta sigma_p), delta = sqrt(2 nu_p / (omega sigma_p)) at the
 * frequency of the next ect_assemble.  h_tet_plate: uint8[n_tets] (host,
 * copied); NULL clears the condition.  The matrix and preconditioner of
 * `which` must be assembled and set up again.  With the condition set,
 * Delta Z is the coil-EMF difference (ect_delta_z needs d_b; ect_impedance
 * does this itself).  ect_set_defect clears a condition set on ECT_DEFECT. */
int ect_set_ibc(ect_ctx* ctx, int which, const uint8_t* h_tet_plate, double sigma_p, double nu_p);

/* Frequency (Hz), nu_tilde = 1/mu_tilde of the Coulomb-gauge penalty (Eq. CGCdiv
 * text) and the V-gauge penalty factor delta of Sec. 4 (1/m^2). */
int ect_set_physics(ect_ctx* ctx, double freq_hz, double nu_tilde, double delta_gauge);

/* Step 3-4 of Sec. 3: assemble the matrix of configuration `which` from the
 * element forms L11, L12, L21, L22 (Sec. 2-3, the coupled form after scaling the
 * V equation by -1/(i omega), with the -i omega sigma mass term in L11 and the
 * delta sigma V gauge penalty in L22), race-free into 4x4 complex blocks (BSR),
 * eliminate A.n = 0, set identity V rows at nodes outside the conductor, and
 * build the symmetric diagonal scaling.  precision_mask (ECT_F64|ECT_F32)
 * selects the scaled copies kept for the solver (F64 is always built). */
int ect_assemble(ect_ctx* ctx, int which, int precision_mask);

/* Subdomain-block preconditioner (the paper's partition of Sec. 3 re-expressed
 * as one dense block per subdomain): inverts the diagonal blocks of the scaled
 * matrix over each subdomain.  precision_mask as for ect_assemble.
 * coarse_group > 0 adds the conductor-V coarse space (two-level, additive):
 * one coarse unknown per group of coarse_group consecutive subdomains that
 * contains a conducting node, V = 1 on that group's conducting nodes (after
 * the per-component gauge freedom of V noted in Sec. 4); its Galerkin matrix
 * is inverted densely (coarse spaces above 16384 unknowns are rejected with
 * ECT_ERR_ARG).  0 = block-Jacobi only.  -1 = aggregation multigrid: the
 * subdomains are the smoothing blocks and the aggregates of the first
 * coarsening (4 coarse unknowns each, Galerkin coarse operators built from
 * the constant field per component), deeper levels aggregate greedily up to
 * 8 nodes, the coarsest level (<= 2048 unknowns) is inverted densely, and each
 * application is one W-cycle with one block-Jacobi sweep before and after the
 * coarse corrections. */
int ect_precond_setup(ect_ctx* ctx, int which, int precision_mask, int coarse_group);

/* Cut every subdomain of the mesh into `parts` (1, 2 or 4) contiguous
 * smoothing blocks of near-equal size: the blocks of the block-Jacobi sweeps
 * and the first aggregates of the multigrid hierarchy (the subdomain size s
 * of the preconditioner).  Every preconditioner must be set up again
 * (ect_precond_setup).  1 = the mesh's subdomains (the default). */
int ect_set_block_split(ect_ctx* ctx, int parts);
int ect_get_block_split(const ect_ctx* ctx);

/* Sizes of the assembled pattern: rows = n_nodes block rows, nnzb blocks. */
int ect_matrix_info(const ect_ctx* ctx, int64_t* n_block_rows, int64_t* nnzb);

/* Copy the assembled, constrained, unscaled FP64 matrix of `which` to the host:
 * h_row_ptr int32[n+1], h_col int32[nnzb], h_val double[nnzb][4][4][2]
 * (block row-major: [row comp][col comp]).  Any pointer may be NULL. */
int ect_matrix_copy(ect_ctx* ctx, int which, int32_t* h_row_ptr, int32_t* h_col, double* h_val);

/* Copy the scaling vector t (double[4*n_nodes]), S = diag(t) M diag(t). */
int ect_scaling_copy(ect_ctx* ctx, int which, double* h_t);

/* y = M x for k vectors (unscaled matrix, FP64), or y = S x with the FP32
 * copy of the scaled matrix S = T M T when precision == ECT_F32 (d_x, d_y
 * complex64; the shared-memory-staged kernel with the default row tiling).
 * d_x, d_y: [k][n_nodes][4], must not overlap. */
int ect_spmv(ect_ctx* ctx, int which, int precision, const void* d_x, void* d_y, int k);

/* Row tiling of the shared-memory-staged FP32 SpMM used by the kernel-level
 * calls ect_spmv (ECT_F32) and ect_precond_apply (ECT_F32, multigrid
 * preconditioner): rows block rows per tile (0 = auto, 32; at most 64);
 * -1 = one thread per scalar row; -2 = one warp per block row.  Solves take
 * ect_options.spmm_rows instead. */
int ect_set_spmm_rows(ect_ctx* ctx, int rows);

/* z = P^-1 r on the scaled system for k vectors ([k][n][4]): the
 * preconditioner set up by ect_precond_setup (subdomain blocks, two-level or
 * multigrid W-cycle). */
int ect_precond_apply(ect_ctx* ctx, int which, int precision, const void* d_r, void* d_z, int k);

/* Classical Gram-Schmidt applied twice (the Arnoldi step of GMRES):
 * d_V holds j orthonormal complex vectors of length n (d_V[i*n + e]),
 * d_w one vector that is overwritten by its projection off span(V);
 * h_h receives the j accumulated coefficients (complex128) and *h_beta the
 * norm of the result.  precision selects complex128 or complex64 storage. */
int ect_cgs2(ect_ctx* ctx, int precision, const void* d_V, int j, int64_t n, void* d_w,
             double* h_h, double* h_beta);

/* Step 6 source term: load vectors of one coil at k probe positions
 * (Sec. 3: mass matrix times the interpolated J of Sec. 4, restricted to the
 * coil, each tet weighted by its volume fraction in the coil).
 * h_z_probe double[k]; d_rhs complex128 [k][n_nodes][4] (V rows zero,
 * constrained dofs zero). */
int ect_coil_rhs(ect_ctx* ctx, const ect_coil* coil, const double* h_z_probe, int k, void* d_rhs);

/* Step 5-6: solve M x = b for k right-hand sides of configuration `which`
 * with preconditioned flexible GMRES (or the mixed FP64/FP32 scheme).
 * d_rhs, d_x complex128 [k][n_nodes][4]; d_x need not be initialised unless
 * opt->x0 = 1, in which case it holds the initial guess.
 * Needs ect_assemble and ect_precond_setup (with ECT_F32 for mixed mode). */
int ect_solve(ect_ctx* ctx, int which, const void* d_rhs, void* d_x, int k,
              const ect_options* opt, ect_stats* stats);

/* Autotuner for batched solves of `which` with k right-hand sides d_rhs
 * (complex128 [k][n_nodes][4]): times the SpMM and preconditioner right-hand-
 * side tile (1, 2, 4, 8) with CUDA events, in mixed mode also the FP32 SpMM
 * variant and row tiling (spmm_rows 32, 24, 16, -1, -2), then runs full solves of d_rhs for
 * each (restart, inner_iters) candidate of the mode in *base and keeps the
 * fastest that converges; in mixed mode the winner is also tried with reorth
 * = 2 and 3; last, the subdomains are cut into 1 and 2 smoothing blocks
 * (ect_set_block_split) with the preconditioner rebuilt and the winner's
 * solve timed again.  *best receives *base with rhs_tile, spmm_rows, restart,
 * inner_iters and reorth replaced; the best subdomain split stays applied to
 * the context (ect_get_block_split) and every preconditioner that was set up
 * before the call is set up again for it.  Stats of the winning solve go to
 * *stats (may be NULL).
 * d_work: complex128 [k][n_nodes][4] scratch for the solutions.  Costs one
 * full solve per candidate; call it once per workload. */
int ect_autotune(ect_ctx* ctx, int which, const void* d_rhs, void* d_work, int k, const ect_options* base,
                 ect_options* best, ect_stats* stats);

/* Eq. impedkl read as the discrete reciprocity identity:
 *   dZ_kl = (i omega / (I_k I_l)) u_k^0^T (M_d - M_0) u_l^d,
 * reduced over the defect tets.  d_u0, d_ud complex128 [2][n_nodes][4] (coil
 * 1 and 2 solutions of the vacuum and defect systems); h_current[2] the coil
 * currents; h_dz receives complex128 [2][2].  If h_dz_emf is not NULL it
 * receives the coil-EMF difference -(i omega/(I_k I_l)) b_k^T (u_l^d - u_l^0)
 * computed from d_b (complex128 [2][n_nodes][4]) as a cross-check.  With an
 * impedance boundary condition (ect_set_ibc) h_dz receives the EMF form and
 * d_b is required. */
int ect_delta_z(ect_ctx* ctx, const void* d_u0, const void* d_ud, const void* d_b,
                const double* h_current, double* h_dz, double* h_dz_emf);

/* The Delta Z reduction of ect_delta_z for n_pos positions (d_u0, d_ud, d_b:
 * complex128 [n_pos][2][n_nodes][4]; h_dz, h_dz_emf: complex128 [n_pos][2][2])
 * that allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 * The paper has no counterpart; this is for callers that cannot allocate
 * device memory, e.g. an application whose device memory is owned by its own
 * pool, or one that must not pay the allocator's latency or the device
 * synchronisation of cudaFree in the middle of its stream work.
 * Scratch: a static device array of 2.1 MB holding partial sums for at most
 * 64 positions (n_pos > 64 returns ECT_ERR_ARG); every GPU that loads the
 * library keeps it until the process exits.  The first call on a device looks
 * up the array's device address (with that device current) and keeps it for
 * the life of the process; make that first call on each device before any
 * stream capture begins.  cudaDeviceReset invalidates the kept address: do
 * not call this function on a device after resetting it.  All calls share
 * the array: calls that overlap on the GPU race.  Synchronises the context
 * stream. */
int ect_delta_z_static(ect_ctx* ctx, const void* d_u0, const void* d_ud, const void* d_b, const double* h_current,
                       int n_pos, double* h_dz, double* h_dz_emf);

/* Step 6-7 for a probe scan: for each of n_pos positions build both coils'
 * sources, solve the vacuum and defect systems (4 solves per position,
 * batched), and reduce Delta Z.  h_dz receives complex128 [n_pos][2][2].
 * Needs both matrices assembled and their preconditioners set up. */
int ect_impedance(ect_ctx* ctx, const ect_coil coils[2], const double* h_z_pos, int n_pos,
                  const ect_options* opt, double* h_dz, ect_stats* stats);

/* ---- frequency sweeps (frequency as a batch dimension) ---------------------
 * Eq. impedmod's signals are read over frequency; the matrices of both
 * configurations change with omega (the -i omega sigma mass term, the
 * -(sigma / (i omega)) V terms and an impedance boundary condition) while
 * the pattern, the coefficients and the constraints do not. */

/* Matrix index of configuration `config` (ECT_VACUUM / ECT_DEFECT) at sweep
 * frequency f; usable as `which` in ect_precond_setup, ect_matrix_copy,
 * ect_scaling_copy, ect_spmv, ect_precond_apply and ect_solve. */
#define ECT_SWEEP_MATRIX(f, config) (2 + 2 * (f) + (config))

/* Assemble both configurations at n_freq (1..16) frequencies h_freq_hz (Hz)
 * in one pass over the pattern per configuration (one kernel writes the
 * n_freq value sets), with the context's coefficients, nu_tilde, delta and
 * impedance boundary condition.  Replaces a previous sweep.  Each sweep
 * matrix then needs ect_precond_setup.  ect_set_mesh, ect_set_physics,
 * ect_set_defect and ect_set_ibc discard the sweep. */
int ect_assemble_sweep(ect_ctx* ctx, const double* h_freq_hz, int n_freq, int precision_mask);

/* Solve configuration `config` at every sweep frequency in one lockstep
 * Krylov solve: d_rhs, d_x complex128 [n_freq][k][n_nodes][4] (block f uses
 * the matrix of frequency f); k * n_freq <= 4096.  Options and statistics as
 * for ect_solve (stats cover all n_freq * k right-hand sides). */
int ect_solve_sweep(ect_ctx* ctx, int config, const void* d_rhs, void* d_x, int k, const ect_options* opt,
                    ect_stats* stats);

/* ect_impedance at every sweep frequency: h_dz receives complex128
 * [n_freq][n_pos][2][2] (Delta Z at each frequency; Z_FA and Z_F3 of
 * Eq. impedmod follow from it).  The coil sources are built once (they do
 * not depend on the frequency) and both configurations are solved for all
 * frequencies in lockstep. */
int ect_impedance_sweep(ect_ctx* ctx, const ect_coil coils[2], const double* h_z_pos, int n_pos,
                        const ect_options* opt, double* h_dz, ect_stats* stats);

/* ---- surrogate MLP ----------------------------------------------------------
 * Not in the paper: a learned map from deposit parameters to the Delta Z
 * signal along the probe path, trained on solver output.  Architecture
 * 6 -> 256 -> 256 -> 256 -> 256 -> 256, SiLU hidden activations, linear
 * output; bf16 weights and activations on tcgen05 tensor cores with fp32
 * accumulation; fp32 master weights and Adam (beta1 0.9, beta2 0.999,
 * eps 1e-8); loss L = 1/(2 B D) sum (y - t)^2.
 * Parameters (float, ect_mlp_num_params() of them): for each layer in order,
 * W (out x in, row-major) then b (out).
 * x: float [batch][6], y/t: float [batch][256], device pointers. */
typedef struct ect_mlp ect_mlp;
int ect_mlp_num_params(void);
/* batch: multiple of 128 (of 256 above 256). */
int ect_mlp_create(ect_mlp** out, void* cuda_stream, int batch);
void ect_mlp_destroy(ect_mlp* m);
const char* ect_mlp_last_error(const ect_mlp* m);
/* Set the fp32 parameters (host) and reset the Adam state. */
int ect_mlp_set_params(ect_mlp* m, const float* h_params);
int ect_mlp_get_params(ect_mlp* m, float* h_params);
/* y = MLP(x) for one batch. */
int ect_mlp_forward(ect_mlp* m, const float* d_x, float* d_y);
/* Loss and its gradient with respect to every parameter (host, same layout). */
int ect_mlp_gradients(ect_mlp* m, const float* d_x, const float* d_t, float* h_grads, double* h_loss);
/* One Adam step on the batch (x, t); *h_loss (if not NULL) receives the loss
 * before the step, which synchronises the stream. */
int ect_mlp_train_step(ect_mlp* m, const float* d_x, const float* d_t, float lr, double* h_loss);

#ifdef __cplusplus
}
#endif

#endif /* ECT_H */
