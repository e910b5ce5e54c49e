// C ABI of the eddy-current solver (declarations and contracts in include/ect.h).
// Every entry point converts exceptions into a status code and a message.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace {
thread_local std::string g_thread_err = "no error";

template <typename F>
int guarded(ect_ctx* c, F&& f) {
    try {
        f();
        if (c) c->err.clear();
        return ECT_OK;
    } catch (const EctError& e) {
        if (c) c->err = e.msg;
        else g_thread_err = e.msg;
        return e.code;
    } catch (const std::exception& e) {
        if (c) c->err = e.what();
        else g_thread_err = e.what();
        return ECT_ERR_ARG;
    } catch (...) {
        if (c) c->err = "unknown error";
        else g_thread_err = "unknown error";
        return ECT_ERR_ARG;
    }
}

void check_which(const ect_ctx* c, int which) {
    ECT_REQUIRE(which_valid(c, which), ECT_ERR_ARG,
                "which must be ECT_VACUUM, ECT_DEFECT or a sweep matrix (ECT_SWEEP_MATRIX)");
}
}  // namespace

int guarded_call(ect_ctx* c, const std::function<void()>& f) { return guarded(c, f); }

extern "C" {

void ect_default_options(ect_options* o) {
    if (!o) return;
    o->tol = 1e-10;
    o->restart = 30;
    o->max_iters = 20000;
    o->mode = ECT_MODE_F64;
    o->inner_iters = 30;
    o->use_graph = 1;
    o->rhs_tile = 0;
    o->timeout_s = 0.0;
    o->reorth = 1;
    o->spmm_rows = 0;
    o->x0 = 0;
}

int ect_create(ect_ctx** out, void* stream) {
    return guarded(nullptr, [&] {
        ECT_REQUIRE(out, ECT_ERR_ARG, "null out pointer");
        *out = nullptr;
        ect_ctx* c = new ect_ctx();
        try {
            ECT_CUDA(cudaGetDevice(&c->device));
            c->stream = (cudaStream_t)stream;
            ECT_CUDA(cudaEventCreate(&c->ev0));
            ECT_CUDA(cudaEventCreate(&c->ev1));
        } catch (...) {
            delete c;
            throw;
        }
        *out = c;
    });
}

void ect_destroy(ect_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    workspace_free(c);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    delete c;
}

const char* ect_last_error(const ect_ctx* c) {
    if (!c) return g_thread_err.c_str();
    return c->err.empty() ? "no error" : c->err.c_str();
}

int ect_set_mesh(ect_ctx* c, const double* xyz, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                 const double* sigma, const double* nu, const double* sigma_d, const double* nu_d,
                 const int32_t* block_of_node, const uint8_t* bc_mask) {
    if (!c) return ECT_ERR_ARG;
    return guarded(c, [&] {
        mesh_setup(c, xyz, n_nodes, tets, n_tets, sigma, nu, sigma_d, nu_d, block_of_node, bc_mask);
    });
}

int ect_partition(const double* xyz, int64_t n_nodes, int max_block_nodes, int32_t* new_id, int32_t* block_of_new) {
    return guarded(nullptr, [&] { partition_rcb(xyz, n_nodes, max_block_nodes, new_id, block_of_new); });
}

int ect_set_defect(ect_ctx* c, const double* sigma_d, const double* nu_d) {
    if (!c) return ECT_ERR_ARG;
    return guarded(c, [&] { set_defect(c, sigma_d, nu_d); });
}

int ect_set_ibc(ect_ctx* c, int which, const uint8_t* plate, double sigma_p, double nu_p) {
    if (!c) return ECT_ERR_ARG;
    return guarded(c, [&] { set_ibc(c, which, plate, sigma_p, nu_p); });
}

int ect_set_physics(ect_ctx* c, double freq, double nu_tilde, double delta) {
    if (!c) return ECT_ERR_ARG;
    return guarded(c, [&] {
        ECT_REQUIRE(std::isfinite(freq) && freq > 0.0, ECT_ERR_ARG, "frequency must be > 0");
        ECT_REQUIRE(std::isfinite(nu_tilde) && nu_tilde >= 0.0, ECT_ERR_ARG, "nu_tilde must be >= 0");
        ECT_REQUIRE(std::isfinite(delta) && delta >= 0.0, ECT_ERR_ARG, "delta must be >= 0");
        c->freq = freq;
        c->omega = 2.0 * 3.14159265358979323846 * freq;
        c->nu_tilde = nu_tilde;
        c->delta = delta;
        c->physics_set = true;
        clear_sweep(c);
        for (int m = 0; m < 2; ++m) c->mat[m].assembled = c->mat[m].pc_f64 = c->mat[m].pc_f32 = false;
    });
}

int ect_assemble(ect_ctx* c, int which, int precision_mask) {
    if (!c) return ECT_ERR_ARG;
    return guarded(c, [&] {
        workspace_free(c);
        assemble_matrix(c, which, precision_mask);
        ECT_CUDA(cudaStreamSynchronize(c->stream));
    });
}

int ect_precond_setup(ect_ctx* c, int which, int precision_mask, int coarse_group) {
    if (!c) return ECT_ERR_ARG;
    return guarded(c, [&] {
        workspace_free(c);
        precond_setup(c, which, precision_mask, coarse_group);
    });
}

int ect_matrix_info(const ect_ctx* c, int64_t* n_rows, int64_t* nnzb) {
    if (!c) return ECT_ERR_ARG;
    if (!c->mesh_set) return ECT_ERR_STATE;
    if (n_rows) *n_rows = c->n_nodes;
    if (nnzb) *nnzb = c->nnzb;
    return ECT_OK;
}

int ect_matrix_copy(ect_ctx* c, int which, int32_t* h_row_ptr, int32_t* h_col, double* h_val) {
    if (!c) return ECT_ERR_ARG;
    return guarded(c, [&] {
        check_which(c, which);
        ECT_REQUIRE(c->mesh_set, ECT_ERR_STATE, "no mesh");
        cudaStream_t st = c->stream;
        if (h_row_ptr)
            ECT_CUDA(cudaMemcpyAsync(h_row_ptr, c->row_ptr.p, c->row_ptr.bytes, cudaMemcpyDeviceToHost, st));
        if (h_col) ECT_CUDA(cudaMemcpyAsync(h_col, c->col.p, c->col.bytes, cudaMemcpyDeviceToHost, st));
        if (h_val) {
            Matrix& M = ctx_mat(c, which);
            ECT_REQUIRE(M.assembled, ECT_ERR_STATE, "matrix not assembled");
            ECT_CUDA(cudaMemcpyAsync(h_val, M.val.p, M.val.bytes, cudaMemcpyDeviceToHost, st));
        }
        ECT_CUDA(cudaStreamSynchronize(st));
    });
}

int ect_scaling_copy(ect_ctx* c, int which, double* h_t) {
    if (!c) return ECT_ERR_ARG;
    return guarded(c, [&] {
        check_which(c, which);
        ECT_REQUIRE(h_t, ECT_ERR_ARG, "null h_t");
        Matrix& M = ctx_mat(c, which);
        ECT_REQUIRE(M.assembled, ECT_ERR_STATE, "matrix not assembled");
        ECT_CUDA(cudaMemcpyAsync(h_t, M.t.p, M.t.bytes, cudaMemcpyDeviceToHost, c->stream));
        ECT_CUDA(cudaStreamSynchronize(c->stream));
    });
}

int ect_spmv(ect_ctx* c, int which, int precision, const void* d_x, void* d_y, int k) {
    if (!c) return ECT_ERR_ARG;
    return guarded(c, [&] {
        check_which(c, which);
        ECT_REQUIRE(d_x && d_y && k >= 1 && k <= 65535, ECT_ERR_ARG, "bad spmv arguments");
        ECT_REQUIRE(d_x != d_y, ECT_ERR_ARG, "x and y must not overlap");
        const int64_t ld = 4 * c->n_nodes;
        if (precision == ECT_F64) spmv_f64(c, which, false, (const double2*)d_x, (double2*)d_y, k, ld, 0, nullptr);
        else if (precision == ECT_F32) {
            c->staged_rows = c->kernel_rows;
            staged_prepare(c, which);
            spmv_f32(c, which, (const float2*)d_x, (float2*)d_y, k, ld, 0, nullptr);
            ECT_REQUIRE(!staged_take_error(c->stream), ECT_ERR_TIMEOUT,
                        "a bounded wait for a bulk copy expired in the staged SpMM");
        }
        else throw EctError{ECT_ERR_ARG, "bad precision"};
    });
}

int ect_set_spmm_rows(ect_ctx* c, int rows) {
    if (!c) return ECT_ERR_ARG;
    return guarded(c, [&] {
        ECT_REQUIRE(rows >= -2 && rows <= 64, ECT_ERR_ARG, "rows must be -2, -1 or in [0, 64]");
        c->kernel_rows = rows == 0 ? STAGED_ROWS_DEFAULT : rows;
    });
}

int ect_precond_apply(ect_ctx* c, int which, int precision, const void* d_r, void* d_z, int k) {
    if (!c) return ECT_ERR_ARG;
    return guarded(c, [&] {
        check_which(c, which);
        ECT_REQUIRE(d_r && d_z && k >= 1 && k <= 65535, ECT_ERR_ARG, "bad precond arguments");
        ECT_REQUIRE(d_r != d_z, ECT_ERR_ARG, "r and z must not overlap");
        const int64_t ld = 4 * c->n_nodes;
        coarse_scratch(c, which, k);
        if (precision == ECT_F64) precond_apply_f64(c, which, (const double2*)d_r, (double2*)d_z, k, ld, 0, nullptr);
        else if (precision == ECT_F32) {
            c->staged_rows = c->kernel_rows;
            staged_prepare(c, which);
            precond_apply_f32(c, which, (const float2*)d_r, (float2*)d_z, k, ld, 0, nullptr);
            ECT_REQUIRE(!staged_take_error(c->stream), ECT_ERR_TIMEOUT,
                        "a bounded wait for a bulk copy expired in the staged SpMM");
        }
        else throw EctError{ECT_ERR_ARG, "bad precision"};
    });
}

int ect_cgs2(ect_ctx* c, int precision, const void* d_V, int j, int64_t n, void* d_w, double* h_h, double* h_beta) {
    if (!c) return ECT_ERR_ARG;
    return guarded(c, [&] { cgs2_entry(c, precision, d_V, j, n, d_w, h_h, h_beta); });
}

int ect_coil_rhs(ect_ctx* c, const ect_coil* coil, const double* h_z_probe, int k, void* d_rhs) {
    if (!c) return ECT_ERR_ARG;
    return guarded(c, [&] {
        ECT_REQUIRE(coil, ECT_ERR_ARG, "null coil");
        coil_rhs(c, *coil, h_z_probe, k, (double2*)d_rhs);
    });
}

int ect_solve(ect_ctx* c, int which, const void* d_rhs, void* d_x, int k, const ect_options* opt, ect_stats* st) {
    if (!c) return ECT_ERR_ARG;
    return guarded(c, [&] {
        ect_options o;
        if (opt) o = *opt;
        else ect_default_options(&o);
        solve(c, which, (const double2*)d_rhs, (double2*)d_x, k, o, st);
    });
}

int ect_autotune(ect_ctx* c, int which, const void* d_rhs, void* d_work, int k, const ect_options* base,
                 ect_options* best, ect_stats* stats) {
    if (!c) return ECT_ERR_ARG;
    return guarded(c, [&] {
        check_which(c, which);
        ECT_REQUIRE(d_rhs && d_work && best && k >= 1, ECT_ERR_ARG, "bad autotune arguments");
        ect_options o;
        if (base) o = *base;
        else ect_default_options(&o);
        o.x0 = 0;  // the solution buffers are this call's own
        Matrix& M = ctx_mat(c, which);
        ECT_REQUIRE(M.assembled && M.pc_f64, ECT_ERR_STATE, "assemble and set up the preconditioner first");
        const bool mixed = o.mode == ECT_MODE_MIXED;
        ECT_REQUIRE(!mixed || (M.has_f32 && M.pc_f32), ECT_ERR_STATE, "mixed mode needs the FP32 operators");
        cudaStream_t st = c->stream;
        const int64_t ld = 4 * c->n_nodes;
        coarse_scratch(c, which, k);
        // 1. kernel tile: SpMM + preconditioner apply on the solver's precision
        DevBuf a, b;
        const size_t esz = mixed ? sizeof(float2) : sizeof(double2);
        a.alloc(esz * ld * k);
        b.alloc(esz * ld * k);
        ECT_CUDA(cudaMemsetAsync(a.p, 0, a.bytes, st));
        int best_tile = 1;
        float best_ms = 1e30f;
        for (int kt : {8, 4, 2, 1, -1}) {
            if (kt > 1 && kt > 2 * k) continue;
            auto run = [&] {
                if (mixed) {
                    spmv_f32(c, which, a.as<float2>(), b.as<float2>(), k, ld, kt, nullptr);
                    precond_apply_f32(c, which, b.as<float2>(), a.as<float2>(), k, ld, kt, nullptr);
                } else {
                    spmv_f64(c, which, true, a.as<double2>(), b.as<double2>(), k, ld, kt, nullptr);
                    precond_apply_f64(c, which, b.as<double2>(), a.as<double2>(), k, ld, kt, nullptr);
                }
            };
            run();
            ECT_CUDA(cudaEventRecord(c->ev0, st));
            for (int r = 0; r < 5; ++r) run();
            ECT_CUDA(cudaEventRecord(c->ev1, st));
            ECT_CUDA(cudaEventSynchronize(c->ev1));
            float ms = 0.f;
            ECT_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
            if (ms < best_ms) {
                best_ms = ms;
                best_tile = kt;
            }
        }
        o.rhs_tile = best_tile;
        // 1b. FP32 SpMM variant and row tiling (mixed mode): the Krylov product plus one
        //     preconditioner application, each candidate with its plans built
        if (mixed) {
            float best_rows_ms = 1e30f;
            int best_rows = o.spmm_rows;
            for (int rows : {0, 24, 16, -1, -2}) {
                c->staged_rows = rows == 0 ? STAGED_ROWS_DEFAULT : rows;
                staged_prepare(c, which);
                auto run = [&] {
                    spmv_f32(c, which, a.as<float2>(), b.as<float2>(), k, ld, o.rhs_tile, nullptr);
                    precond_apply_f32(c, which, b.as<float2>(), a.as<float2>(), k, ld, o.rhs_tile, nullptr);
                };
                run();
                ECT_CUDA(cudaEventRecord(c->ev0, st));
                for (int r = 0; r < 5; ++r) run();
                ECT_CUDA(cudaEventRecord(c->ev1, st));
                ECT_CUDA(cudaEventSynchronize(c->ev1));
                float ms = 0.f;
                ECT_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
                if (ms < best_rows_ms) {
                    best_rows_ms = ms;
                    best_rows = rows;
                }
            }
            ECT_REQUIRE(!staged_take_error(st), ECT_ERR_TIMEOUT,
                        "a bounded wait for a bulk copy expired in the staged SpMM");
            o.spmm_rows = best_rows;
        }
        // 2. Krylov lengths: full solves, fastest converged wins
        std::vector<std::pair<int, int>> cand;
        if (mixed) cand = {{10, 10}, {10, 20}, {8, 30}, {16, 12}, {16, 16}, {12, 24}, {16, 20}, {16, 24}};
        else cand = {{20, 0}, {30, 0}, {45, 0}};
        double best_t = 1e300;
        ect_options win = o;
        ect_stats wst{};
        bool any = false;
        for (auto& pr : cand) {
            ect_options t = o;
            t.restart = pr.first;
            if (mixed) t.inner_iters = pr.second;
            ect_stats s{};
            try {
                solve(c, which, (const double2*)d_rhs, (double2*)d_work, k, t, &s);
            } catch (const EctError& e) {
                if (e.code != ECT_ERR_NOT_CONVERGED && e.code != ECT_ERR_TIMEOUT) throw;
                continue;
            }
            if (s.ms < best_t) {
                best_t = s.ms;
                win = t;
                wst = s;
                any = true;
            }
        }
        ECT_REQUIRE(any, ECT_ERR_NOT_CONVERGED, "no autotune candidate converged");
        if (mixed) {
            // the winner again with one Gram-Schmidt pass in the FP32 loop (2), then in both loops (3)
            const ect_options w0 = win;
            for (int ro : {2, 3}) {
                if (w0.reorth == ro) continue;
                ect_options t = w0;
                t.reorth = ro;
                ect_stats s{};
                try {
                    solve(c, which, (const double2*)d_rhs, (double2*)d_work, k, t, &s);
                    if (s.ms < best_t) {
                        best_t = s.ms;
                        win = t;
                        wst = s;
                    }
                } catch (const EctError& e) {
                    if (e.code != ECT_ERR_NOT_CONVERGED && e.code != ECT_ERR_TIMEOUT) throw;
                }
            }
        }
        // 3. subdomain size: each subdomain cut into `parts` smoothing blocks (also the first
        //    multigrid aggregates), the preconditioner rebuilt, the winner's solve timed again
        {
            const int n_mat = 2 + (int)c->smat.size();
            std::vector<char> had(n_mat, 0);
            for (int m = 0; m < n_mat; ++m) had[m] = ctx_mat(c, m).pc_f64;
            const int start = c->block_split;
            int best_parts = start;
            for (int parts : {1, 2}) {
                if (parts == start) continue;
                set_block_split(c, parts);
                precond_setup(c, which, M.pc_mask, M.pc_group);
                coarse_scratch(c, which, k);
                ect_stats s{};
                try {
                    solve(c, which, (const double2*)d_rhs, (double2*)d_work, k, win, &s);
                    if (s.ms < best_t) {
                        best_t = s.ms;
                        best_parts = parts;
                        wst = s;
                    }
                } catch (const EctError& e) {
                    if (e.code != ECT_ERR_NOT_CONVERGED && e.code != ECT_ERR_TIMEOUT) throw;
                }
            }
            if (c->block_split != best_parts || best_parts != start) {
                set_block_split(c, best_parts);
                for (int m = 0; m < n_mat; ++m)
                    if (had[m] || m == which) {
                        Matrix& Mm = ctx_mat(c, m);
                        precond_setup(c, m, Mm.pc_mask, Mm.pc_group);
                    }
            }
        }
        *best = win;
        if (stats) *stats = wst;
    });
}

int ect_set_block_split(ect_ctx* c, int parts) {
    if (!c) return ECT_ERR_ARG;
    return guarded(c, [&] { set_block_split(c, parts); });
}

int ect_get_block_split(const ect_ctx* c) { return c ? c->block_split : 0; }

int ect_assemble_sweep(ect_ctx* c, const double* freq_hz, int n_freq, int precision_mask) {
    if (!c) return ECT_ERR_ARG;
    return guarded(c, [&] { assemble_sweep(c, freq_hz, n_freq, precision_mask); });
}

int ect_solve_sweep(ect_ctx* c, int config, const void* d_rhs, void* d_x, int k, const ect_options* opt,
                    ect_stats* st) {
    if (!c) return ECT_ERR_ARG;
    return guarded(c, [&] {
        ect_options o;
        if (opt) o = *opt;
        else ect_default_options(&o);
        solve_sweep(c, config, (const double2*)d_rhs, (double2*)d_x, k, o, st);
    });
}

int ect_impedance_sweep(ect_ctx* c, const ect_coil coils[2], const double* h_z_pos, int n_pos,
                        const ect_options* opt, double* h_dz, ect_stats* stats) {
    if (!c) return ECT_ERR_ARG;
    return guarded(c, [&] {
        ECT_REQUIRE(coils && h_z_pos && h_dz && n_pos >= 1, ECT_ERR_ARG, "bad impedance arguments");
        const int F = (int)c->sweep_omega.size();
        ECT_REQUIRE(F >= 1, ECT_ERR_STATE, "no frequency sweep assembled (ect_assemble_sweep)");
        for (int m = 2; m < 2 + 2 * F; ++m)
            ECT_REQUIRE(ctx_mat(c, m).assembled && ctx_mat(c, m).pc_f64, ECT_ERR_STATE,
                        "set up the preconditioner of every sweep matrix first");
        ect_options o;
        if (opt) o = *opt;
        else ect_default_options(&o);
        o.x0 = 0;  // the solution buffers are this call's own
        const int64_t nvec = 4 * c->n_nodes;
        size_t fr = 0, tot = 0;
        ECT_CUDA(cudaMemGetInfo(&fr, &tot));
        const int m = o.restart, mi = o.mode == ECT_MODE_MIXED ? o.inner_iters : 0;
        const double per_rhs = (double)nvec * F * (16.0 * (2 * m + 8) + 8.0 * (mi + 2));
        int chunk = (int)std::max(1.0, std::min<double>(n_pos, 0.5 * (double)fr / (2.0 * per_rhs)));
        chunk = std::min(chunk, std::max(1, 2048 / (2 * F)));
        DevBuf B, U0, Ud;
        B.alloc(sizeof(double2) * nvec * 2 * chunk);            // sources: the same at every frequency
        U0.alloc(sizeof(double2) * nvec * 2 * chunk * F);       // [F][2 chunk][4N]
        Ud.alloc(U0.bytes);
        const double cur[2] = {coils[0].J_e * (coils[0].r_out - coils[0].r_in) * coils[0].length,
                               coils[1].J_e * (coils[1].r_out - coils[1].r_in) * coils[1].length};
        ect_stats agg{};
        std::vector<double> dz(8 * (size_t)chunk);
        for (int p0 = 0; p0 < n_pos; p0 += chunk) {
            const int np = std::min(chunk, n_pos - p0);
            for (int cc = 0; cc < 2; ++cc) {
                DevBuf tmp;
                tmp.alloc(sizeof(double2) * nvec * np);
                coil_rhs(c, coils[cc], h_z_pos + p0, np, tmp.as<double2>());
                ECT_CUDA(cudaMemcpy2DAsync(B.as<double2>() + cc * nvec, 2 * nvec * sizeof(double2), tmp.p,
                                           nvec * sizeof(double2), nvec * sizeof(double2), np,
                                           cudaMemcpyDeviceToDevice, c->stream));
            }
            ect_stats s0{}, s1{};
            int rc = ECT_OK;
            for (int cfg = 0; cfg < 2; ++cfg) {
                try {
                    solve_sweep(c, cfg, B.as<double2>(), (cfg ? Ud : U0).as<double2>(), 2 * np, o, cfg ? &s1 : &s0,
                                true);
                } catch (const EctError& e) {
                    if (e.code != ECT_ERR_NOT_CONVERGED) throw;
                    rc = e.code;
                }
            }
            for (int f = 0; f < F; ++f) {
                const int64_t off = (int64_t)f * 2 * np * nvec;
                delta_z(c, U0.as<double2>() + off, Ud.as<double2>() + off, B.as<double2>(), cur, np, dz.data(),
                        nullptr, c->sweep_omega[f]);
                for (int q = 0; q < np; ++q)
                    for (int e = 0; e < 8; ++e) h_dz[((int64_t)f * n_pos + p0 + q) * 8 + e] = dz[(size_t)q * 8 + e];
            }
            agg.iters = std::max({agg.iters, s0.iters, s1.iters});
            agg.outer_iters = std::max({agg.outer_iters, s0.outer_iters, s1.outer_iters});
            agg.converged += s0.converged + s1.converged;
            agg.restarts += s0.restarts + s1.restarts;
            agg.relres_max = std::max({agg.relres_max, s0.relres_max, s1.relres_max});
            agg.ms += s0.ms + s1.ms;
            agg.launches += s0.launches + s1.launches + 4 + F;
            if (rc != ECT_OK) {
                if (stats) *stats = agg;
                throw EctError{ECT_ERR_NOT_CONVERGED, "a probe solve did not reach the tolerance"};
            }
        }
        if (stats) *stats = agg;
    });
}

int ect_delta_z(ect_ctx* c, const void* d_u0, const void* d_ud, const void* d_b, const double* h_current, double* h_dz,
                double* h_dz_emf) {
    if (!c) return ECT_ERR_ARG;
    return guarded(c, [&] {
        delta_z(c, (const double2*)d_u0, (const double2*)d_ud, (const double2*)d_b, h_current, 1, h_dz, h_dz_emf);
    });
}

int ect_impedance(ect_ctx* c, const ect_coil coils[2], const double* h_z_pos, int n_pos, const ect_options* opt,
                  double* h_dz, ect_stats* stats) {
    if (!c) return ECT_ERR_ARG;
    return guarded(c, [&] {
        ECT_REQUIRE(coils && h_z_pos && h_dz && n_pos >= 1, ECT_ERR_ARG, "bad impedance arguments");
        for (int m = 0; m < 2; ++m)
            ECT_REQUIRE(c->mat[m].assembled && c->mat[m].pc_f64, ECT_ERR_STATE,
                        "assemble both matrices and set up their preconditioners first");
        ect_options o;
        if (opt) o = *opt;
        else ect_default_options(&o);
        o.x0 = 0;  // the solution buffers are this call's own
        const int64_t nvec = 4 * c->n_nodes;
        // positions per batch: bounded by the Krylov workspace of 2 rhs per position
        size_t fr = 0, tot = 0;
        ECT_CUDA(cudaMemGetInfo(&fr, &tot));
        const int m = o.restart, mi = o.mode == ECT_MODE_MIXED ? o.inner_iters : 0;
        const double per_rhs = (double)nvec * (16.0 * (2 * m + 8) + 8.0 * (mi + 2));
        int chunk = (int)std::max(1.0, std::min<double>(n_pos, 0.5 * (double)fr / (2.0 * per_rhs)));
        chunk = std::min(chunk, 32);
        DevBuf B, U0, Ud;
        B.alloc(sizeof(double2) * nvec * 2 * chunk);
        U0.alloc(B.bytes);
        Ud.alloc(B.bytes);
        const double cur[2] = {coils[0].J_e * (coils[0].r_out - coils[0].r_in) * coils[0].length,
                               coils[1].J_e * (coils[1].r_out - coils[1].r_in) * coils[1].length};
        ect_stats agg{};
        for (int p0 = 0; p0 < n_pos; p0 += chunk) {
            const int np = std::min(chunk, n_pos - p0);
            for (int cc = 0; cc < 2; ++cc) {
                // coil cc of position p goes to rhs index 2p + cc
                DevBuf tmp;
                tmp.alloc(sizeof(double2) * nvec * np);
                coil_rhs(c, coils[cc], h_z_pos + p0, np, tmp.as<double2>());
                ECT_CUDA(cudaMemcpy2DAsync(B.as<double2>() + cc * nvec, 2 * nvec * sizeof(double2), tmp.p,
                                           nvec * sizeof(double2), nvec * sizeof(double2), np,
                                           cudaMemcpyDeviceToDevice, c->stream));
            }
            ect_stats s0{}, s1{};
            int rc0 = ECT_OK, rc1 = ECT_OK;
            try {
                solve(c, ECT_VACUUM, B.as<double2>(), U0.as<double2>(), 2 * np, o, &s0);
            } catch (const EctError& e) {
                if (e.code != ECT_ERR_NOT_CONVERGED) throw;
                rc0 = e.code;
            }
            try {
                solve(c, ECT_DEFECT, B.as<double2>(), Ud.as<double2>(), 2 * np, o, &s1);
            } catch (const EctError& e) {
                if (e.code != ECT_ERR_NOT_CONVERGED) throw;
                rc1 = e.code;
            }
            delta_z(c, U0.as<double2>(), Ud.as<double2>(), B.as<double2>(), cur, np, h_dz + (int64_t)p0 * 8, nullptr);
            agg.iters = std::max({agg.iters, s0.iters, s1.iters});
            agg.outer_iters = std::max({agg.outer_iters, s0.outer_iters, s1.outer_iters});
            agg.converged += s0.converged + s1.converged;
            agg.restarts += s0.restarts + s1.restarts;
            agg.relres_max = std::max({agg.relres_max, s0.relres_max, s1.relres_max});
            agg.ms += s0.ms + s1.ms;
            agg.launches += s0.launches + s1.launches + 5;  // + 2 coil-source kernels per coil, Delta Z
            if (rc0 != ECT_OK || rc1 != ECT_OK) {
                if (stats) *stats = agg;
                throw EctError{ECT_ERR_NOT_CONVERGED, "a probe solve did not reach the tolerance"};
            }
        }
        if (stats) *stats = agg;
    });
}

}  // extern "C"
