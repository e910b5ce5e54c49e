// Mesh input, tet geometry and the block-sparse (BSR) pattern.
//
// Steps 1-2 of Sec. 3 (triangulation and partition).  The paper's parallel
// assembly sums per-subdomain Morse matrices with an MPI reduction (Sec. 3,
// Steps 3-4); on one GPU that sum becomes an owner-computes gather: every
// 4x4 block (row node i, column node j) of the matrix is produced by one
// thread that walks the list of (tet, local i, local j) triples touching it.
// This file builds that list once per mesh: the per-row lists of all
// (tet, a, b) node pairs, sorted by (column, tet), give both the BSR column
// indices and, for each block, the contiguous run of its contributions.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace {

// vol and barycentric gradients: with rows r_a = x_a - x_0 (a = 1..3) and
// det = r1 . (r2 x r3), grad l_1 = r2 x r3 / det, grad l_2 = r3 x r1 / det,
// grad l_3 = r1 x r2 / det and grad l_0 = -(grad l_1 + grad l_2 + grad l_3).
__global__ void k_tet_geometry(const double* __restrict__ xyz, const int32_t* __restrict__ tets,
                               int64_t n_tets, double* __restrict__ geo, int* __restrict__ bad) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_tets) return;
    double p[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        int n = tets[4 * t + a];
#pragma unroll
        for (int i = 0; i < 3; ++i) p[a][i] = xyz[3 * (int64_t)n + i];
    }
    double r[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) r[a][i] = p[a + 1][i] - p[0][i];
    double c23[3] = {r[1][1] * r[2][2] - r[1][2] * r[2][1], r[1][2] * r[2][0] - r[1][0] * r[2][2],
                     r[1][0] * r[2][1] - r[1][1] * r[2][0]};
    double c31[3] = {r[2][1] * r[0][2] - r[2][2] * r[0][1], r[2][2] * r[0][0] - r[2][0] * r[0][2],
                     r[2][0] * r[0][1] - r[2][1] * r[0][0]};
    double c12[3] = {r[0][1] * r[1][2] - r[0][2] * r[1][1], r[0][2] * r[1][0] - r[0][0] * r[1][2],
                     r[0][0] * r[1][1] - r[0][1] * r[1][0]};
    double det = r[0][0] * c23[0] + r[0][1] * c23[1] + r[0][2] * c23[2];
    double* g = geo + 16 * t;
    if (!(det > 0.0)) {
        atomicExch(bad, 1);
        det = 1.0;
    }
    double inv = 1.0 / det;
    g[0] = det / 6.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        double g1 = c23[i] * inv, g2 = c31[i] * inv, g3 = c12[i] * inv;
        g[1 + 3 + i] = g1;
        g[1 + 6 + i] = g2;
        g[1 + 9 + i] = g3;
        g[1 + i] = -(g1 + g2 + g3);
    }
    g[13] = g[14] = g[15] = 0.0;
}

// each (tet, a) adds 4 pair entries to row tets[t][a]
__global__ void k_count_pairs(const int32_t* __restrict__ tets, int64_t n4, int* __restrict__ cnt) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n4) return;
    atomicAdd(&cnt[tets[e]], 4);
}

__global__ void k_fill_pairs(const int32_t* __restrict__ tets, int64_t n_tets,
                             const int64_t* __restrict__ row_start, int* __restrict__ fill,
                             unsigned long long* __restrict__ keys) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= 4 * n_tets) return;
    int64_t t = e >> 2;
    int a = (int)(e & 3);
    int row = tets[e];
    int pos = atomicAdd(&fill[row], 4);
    int64_t base = row_start[row] + pos;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        unsigned int col = (unsigned int)tets[4 * t + b];
        unsigned int ent = (unsigned int)((t << 4) | (a << 2) | b);
        keys[base + b] = ((unsigned long long)col << 32) | ent;
    }
}

// sort each row's keys (short rows: insertion sort), then count distinct columns
__global__ void k_sort_rows(unsigned long long* __restrict__ keys, const int64_t* __restrict__ row_start,
                            int64_t n_rows, int* __restrict__ n_unique) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    int64_t s = row_start[r], e = row_start[r + 1];
    for (int64_t i = s + 1; i < e; ++i) {
        unsigned long long k = keys[i];
        int64_t j = i - 1;
        while (j >= s && keys[j] > k) {
            keys[j + 1] = keys[j];
            --j;
        }
        keys[j + 1] = k;
    }
    int u = 0;
    unsigned long long prev = ~0ull;
    for (int64_t i = s; i < e; ++i) {
        unsigned long long c = keys[i] >> 32;
        if (c != prev) ++u;
        prev = c;
    }
    n_unique[r] = u;
}

__global__ void k_fill_bsr(const unsigned long long* __restrict__ keys, const int64_t* __restrict__ row_start,
                           int64_t n_rows, const int32_t* __restrict__ row_ptr, int32_t* __restrict__ col,
                           int32_t* __restrict__ slot_ptr, int32_t* __restrict__ diag_slot,
                           uint32_t* __restrict__ entries) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    int64_t s = row_start[r], e = row_start[r + 1];
    int slot = row_ptr[r];
    unsigned long long prev = ~0ull;
    for (int64_t i = s; i < e; ++i) {
        unsigned long long c = keys[i] >> 32;
        if (c != prev) {
            col[slot] = (int32_t)c;
            slot_ptr[slot] = (int32_t)i;
            if ((int64_t)c == r) diag_slot[r] = slot;
            ++slot;
            prev = c;
        }
        entries[i] = (uint32_t)(keys[i] & 0xffffffffull);
    }
}


// per-tet coefficients of the defect configuration (NaN = background)
void defect_coefficients(const std::vector<double>& s0, const std::vector<double>& n0, const double* sigma_d,
                         const double* nu_d, std::vector<double>& s1, std::vector<double>& n1) {
    s1 = s0;
    n1 = n0;
    for (size_t t = 0; t < s0.size(); ++t) {
        if (sigma_d && !std::isnan(sigma_d[t])) {
            ECT_REQUIRE(std::isfinite(sigma_d[t]) && sigma_d[t] >= 0.0, ECT_ERR_ARG, "bad defect sigma");
            s1[t] = sigma_d[t];
        }
        if (nu_d && !std::isnan(nu_d[t])) {
            ECT_REQUIRE(std::isfinite(nu_d[t]) && nu_d[t] > 0.0, ECT_ERR_ARG, "bad defect nu");
            n1[t] = nu_d[t];
        }
    }
}

}  // namespace

// coefficients, conducting nodes and constraint mask of configuration m
void upload_config(ect_ctx* c, int m, const std::vector<double>& s, const std::vector<double>& n) {
    const int64_t N = c->n_nodes, T = c->n_tets;
    Matrix& M = c->mat[m];
    if (&M.h_sigma != &s) M.h_sigma = s;
    if (&M.h_nu != &n) M.h_nu = n;
    const bool plate = M.ibc && (int64_t)M.h_void.size() == T;
    // conducting nodes and (with a plate removed by the IBC) nodes that keep a volume form
    M.h_cond.assign(N, 0);
    std::vector<uint8_t> live(N, plate ? 0 : 1);
    for (int64_t t = 0; t < T; ++t) {
        if (plate && M.h_void[t]) continue;
        for (int a = 0; a < 4; ++a) {
            live[c->h_tets[4 * t + a]] = 1;
            if (s[t] > 0.0) M.h_cond[c->h_tets[4 * t + a]] = 1;
        }
    }
    std::vector<uint8_t> fm(N);
    for (int64_t i = 0; i < N; ++i)
        fm[i] = live[i] ? (uint8_t)((c->h_bc[i] & 7) | (M.h_cond[i] ? 0 : 8)) : (uint8_t)15;  // plate inside: all fixed
    M.h_fix = fm;
    cudaStream_t st = c->stream;
    M.sigma.alloc(sizeof(double) * T);
    M.nu.alloc(sizeof(double) * T);
    M.fixmask.alloc(N);
    ECT_CUDA(cudaMemcpyAsync(M.sigma.p, s.data(), M.sigma.bytes, cudaMemcpyHostToDevice, st));
    ECT_CUDA(cudaMemcpyAsync(M.nu.p, n.data(), M.nu.bytes, cudaMemcpyHostToDevice, st));
    ECT_CUDA(cudaMemcpyAsync(M.fixmask.p, fm.data(), N, cudaMemcpyHostToDevice, st));
    ECT_CUDA(cudaStreamSynchronize(st));
    M.assembled = M.pc_f64 = M.pc_f32 = false;
}

namespace {

// Omega_d: the tets whose coefficients differ between the two configurations
void upload_defect_list(ect_ctx* c, const std::vector<double>& s1, const std::vector<double>& n1) {
    std::vector<int32_t> od;
    for (int64_t t = 0; t < c->n_tets; ++t)
        if (s1[t] != c->h_sigma0[t] || n1[t] != c->h_nu0[t]) od.push_back((int32_t)t);
    c->n_omega_d = (int64_t)od.size();
    c->omega_d.alloc(sizeof(int32_t) * std::max<size_t>(od.size(), 1));
    if (!od.empty())
        ECT_CUDA(cudaMemcpyAsync(c->omega_d.p, od.data(), sizeof(int32_t) * od.size(), cudaMemcpyHostToDevice,
                                 c->stream));
    ECT_CUDA(cudaStreamSynchronize(c->stream));
}

}  // namespace

// The smoothing blocks (and first multigrid aggregates): the mesh's subdomains,
// each cut into c->block_split contiguous pieces of near-equal size.
void apply_block_split(ect_ctx* c) {
    const std::vector<int32_t>& mb = c->h_block_ptr_mesh;
    std::vector<int32_t> bptr(1, 0);
    for (size_t b = 0; b + 1 < mb.size(); ++b) {
        const int n = mb[b + 1] - mb[b];
        const int parts = std::min(c->block_split, n);
        for (int q = 1; q <= parts; ++q) bptr.push_back(mb[b] + (int32_t)((int64_t)n * q / parts));
    }
    int maxb = 0;
    std::vector<int64_t> poff(bptr.size(), 0), poff32(bptr.size(), 0);
    for (size_t b = 0; b + 1 < bptr.size(); ++b) {
        const int sz = bptr[b + 1] - bptr[b];
        maxb = std::max(maxb, sz);
        poff[b + 1] = poff[b] + (int64_t)(4 * sz) * (4 * sz);
        poff32[b + 1] = poff32[b] + sym_packed_size(4 * sz);
    }
    c->n_blocks = (int64_t)bptr.size() - 1;
    c->max_block_nodes = maxb;
    c->h_block_ptr = bptr;
    c->pinv_total = poff.back();
    c->pinv_total32 = poff32.back();
    cudaStream_t st = c->stream;
    c->block_ptr.alloc(sizeof(int32_t) * bptr.size());
    c->pinv_off.alloc(sizeof(int64_t) * poff.size());
    c->pinv_off32.alloc(sizeof(int64_t) * poff32.size());
    ECT_CUDA(cudaMemcpyAsync(c->block_ptr.p, bptr.data(), c->block_ptr.bytes, cudaMemcpyHostToDevice, st));
    ECT_CUDA(cudaMemcpyAsync(c->pinv_off.p, poff.data(), c->pinv_off.bytes, cudaMemcpyHostToDevice, st));
    ECT_CUDA(cudaMemcpyAsync(c->pinv_off32.p, poff32.data(), c->pinv_off32.bytes, cudaMemcpyHostToDevice, st));
    ECT_CUDA(cudaStreamSynchronize(st));
}

void set_block_split(ect_ctx* c, int parts) {
    ECT_REQUIRE(c->mesh_set, ECT_ERR_STATE, "ect_set_mesh must come first");
    ECT_REQUIRE(parts == 1 || parts == 2 || parts == 4, ECT_ERR_ARG, "parts must be 1, 2 or 4");
    if (parts == c->block_split) return;
    workspace_free(c);
    auto invalidate = [](Matrix& M) {
        mg_free(M);
        M.pc_f64 = M.pc_f32 = false;
    };
    for (int m = 0; m < 2; ++m) invalidate(c->mat[m]);
    for (Matrix& M : c->smat) invalidate(M);
    c->block_split = parts;
    apply_block_split(c);
}

void clear_sweep(ect_ctx* c) {
    workspace_free(c);
    c->smat.clear();
    c->sweep_omega.clear();
}

void set_defect(ect_ctx* c, const double* sigma_d, const double* nu_d) {
    ECT_REQUIRE(c->mesh_set, ECT_ERR_STATE, "ect_set_mesh must come first");
    std::vector<double> s1, n1;
    defect_coefficients(c->h_sigma0, c->h_nu0, sigma_d, nu_d, s1, n1);
    clear_sweep(c);
    c->mat[1].reset();
    upload_config(c, 1, s1, n1);
    upload_defect_list(c, s1, n1);
}

void mesh_setup(ect_ctx* c, const double* xyz, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                const double* sigma, const double* nu, const double* sigma_d, const double* nu_d,
                const int32_t* block_of_node, const uint8_t* bc_mask) {
    ECT_REQUIRE(xyz && tets && sigma && nu && block_of_node && bc_mask, ECT_ERR_ARG, "null mesh array");
    ECT_REQUIRE(n_nodes > 0 && n_tets > 0, ECT_ERR_ARG, "empty mesh");
    ECT_REQUIRE(n_nodes < (1ll << 30), ECT_ERR_ARG, "too many nodes (limit 2^30)");
    ECT_REQUIRE(n_tets < (1ll << 27), ECT_ERR_ARG, "too many tets (limit 2^27)");
    for (int64_t e = 0; e < 4 * n_tets; ++e)
        ECT_REQUIRE(tets[e] >= 0 && tets[e] < n_nodes, ECT_ERR_MESH, "tet node index out of range");
    for (int64_t t = 0; t < n_tets; ++t)
        ECT_REQUIRE(std::isfinite(sigma[t]) && std::isfinite(nu[t]) && sigma[t] >= 0.0 && nu[t] > 0.0,
                    ECT_ERR_ARG, "sigma must be finite >= 0 and nu finite > 0");
    // partition: contiguous non-decreasing blocks of at most 16 nodes
    ECT_REQUIRE(block_of_node[0] == 0, ECT_ERR_ARG, "block_of_node must start at 0");
    std::vector<int32_t> bptr(1, 0);
    for (int64_t n = 1; n < n_nodes; ++n) {
        int32_t d = block_of_node[n] - block_of_node[n - 1];
        ECT_REQUIRE(d == 0 || d == 1, ECT_ERR_ARG, "block_of_node must be non-decreasing in steps of 0 or 1");
        if (d == 1) bptr.push_back((int32_t)n);
    }
    bptr.push_back((int32_t)n_nodes);
    int maxb = 0;
    for (size_t b = 0; b + 1 < bptr.size(); ++b) maxb = std::max(maxb, bptr[b + 1] - bptr[b]);
    ECT_REQUIRE(maxb <= 16, ECT_ERR_ARG, "a subdomain block has more than 16 nodes");

    // effective coefficients of the two configurations
    std::vector<double> s0(sigma, sigma + n_tets), n0(nu, nu + n_tets);
    std::vector<double> s1, n1;
    defect_coefficients(s0, n0, sigma_d, nu_d, s1, n1);

    // reset state
    c->mesh_set = false;
    clear_sweep(c);
    for (int m = 0; m < 2; ++m) c->mat[m].reset();
    c->fine_plan.reset();
    c->n_nodes = n_nodes;
    c->n_tets = n_tets;
    c->h_block_ptr_mesh = bptr;
    c->block_split = 1;
    cudaStream_t st = c->stream;

    c->xyz.alloc(sizeof(double) * 3 * n_nodes);
    c->tets.alloc(sizeof(int32_t) * 4 * n_tets);
    c->bc.alloc(n_nodes);
    ECT_CUDA(cudaMemcpyAsync(c->xyz.p, xyz, c->xyz.bytes, cudaMemcpyHostToDevice, st));
    ECT_CUDA(cudaMemcpyAsync(c->tets.p, tets, c->tets.bytes, cudaMemcpyHostToDevice, st));
    ECT_CUDA(cudaMemcpyAsync(c->bc.p, bc_mask, n_nodes, cudaMemcpyHostToDevice, st));
    apply_block_split(c);
    c->h_tets.assign(tets, tets + 4 * n_tets);
    c->h_bc.assign(bc_mask, bc_mask + n_nodes);
    c->h_sigma0 = s0;
    c->h_nu0 = n0;
    upload_config(c, 0, s0, n0);
    upload_config(c, 1, s1, n1);
    upload_defect_list(c, s1, n1);

    // geometry
    c->geo.alloc(sizeof(double) * 16 * n_tets);
    DevBuf flag;
    flag.alloc(sizeof(int));
    ECT_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), st));
    k_tet_geometry<<<grid_for(n_tets, 256), 256, 0, st>>>(c->xyz.as<double>(), c->tets.as<int32_t>(), n_tets,
                                                          c->geo.as<double>(), flag.as<int>());
    ECT_CHECK_LAUNCH();
    int h_bad = 0;
    ECT_CUDA(cudaMemcpyAsync(&h_bad, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    ECT_CUDA(cudaStreamSynchronize(st));
    ECT_REQUIRE(!h_bad, ECT_ERR_MESH, "a tet has non-positive volume (orientation or degenerate)");

    // pattern: per-row pair lists
    DevBuf cnt, rstart, keys, fill, uniq;
    cnt.alloc(sizeof(int) * n_nodes);
    ECT_CUDA(cudaMemsetAsync(cnt.p, 0, cnt.bytes, st));
    k_count_pairs<<<grid_for(4 * n_tets, 256), 256, 0, st>>>(c->tets.as<int32_t>(), 4 * n_tets, cnt.as<int>());
    ECT_CHECK_LAUNCH();
    std::vector<int> hcnt(n_nodes);
    ECT_CUDA(cudaMemcpyAsync(hcnt.data(), cnt.p, cnt.bytes, cudaMemcpyDeviceToHost, st));
    ECT_CUDA(cudaStreamSynchronize(st));
    std::vector<int64_t> hstart(n_nodes + 1, 0);
    for (int64_t n = 0; n < n_nodes; ++n) {
        ECT_REQUIRE(hcnt[n] > 0, ECT_ERR_MESH, "a node belongs to no tet");
        hstart[n + 1] = hstart[n] + hcnt[n];
    }
    int64_t total = hstart[n_nodes];
    rstart.alloc(sizeof(int64_t) * (n_nodes + 1));
    ECT_CUDA(cudaMemcpyAsync(rstart.p, hstart.data(), rstart.bytes, cudaMemcpyHostToDevice, st));
    keys.alloc(sizeof(unsigned long long) * total);
    fill.alloc(sizeof(int) * n_nodes);
    ECT_CUDA(cudaMemsetAsync(fill.p, 0, fill.bytes, st));
    k_fill_pairs<<<grid_for(4 * n_tets, 256), 256, 0, st>>>(c->tets.as<int32_t>(), n_tets, rstart.as<int64_t>(),
                                                            fill.as<int>(), keys.as<unsigned long long>());
    ECT_CHECK_LAUNCH();
    uniq.alloc(sizeof(int) * n_nodes);
    k_sort_rows<<<grid_for(n_nodes, 128), 128, 0, st>>>(keys.as<unsigned long long>(), rstart.as<int64_t>(),
                                                        n_nodes, uniq.as<int>());
    ECT_CHECK_LAUNCH();
    std::vector<int> hu(n_nodes);
    ECT_CUDA(cudaMemcpyAsync(hu.data(), uniq.p, uniq.bytes, cudaMemcpyDeviceToHost, st));
    ECT_CUDA(cudaStreamSynchronize(st));
    std::vector<int32_t> hrp(n_nodes + 1, 0);
    int64_t nnzb = 0;
    for (int64_t n = 0; n < n_nodes; ++n) {
        nnzb += hu[n];
        ECT_REQUIRE(nnzb < (1ll << 31), ECT_ERR_ARG, "too many blocks");
        hrp[n + 1] = (int32_t)nnzb;
    }
    ECT_REQUIRE(total < (1ll << 31), ECT_ERR_ARG, "too many pair entries");
    c->nnzb = nnzb;
    c->n_entries = total;
    c->row_ptr.alloc(sizeof(int32_t) * (n_nodes + 1));
    ECT_CUDA(cudaMemcpyAsync(c->row_ptr.p, hrp.data(), c->row_ptr.bytes, cudaMemcpyHostToDevice, st));
    c->col.alloc(sizeof(int32_t) * nnzb);
    c->slot_ptr.alloc(sizeof(int32_t) * (nnzb + 1));
    c->diag_slot.alloc(sizeof(int32_t) * n_nodes);
    c->entries.alloc(sizeof(uint32_t) * total);
    int32_t tot32 = (int32_t)total;
    ECT_CUDA(cudaMemcpyAsync(c->slot_ptr.as<int32_t>() + nnzb, &tot32, sizeof(int32_t), cudaMemcpyHostToDevice, st));
    k_fill_bsr<<<grid_for(n_nodes, 128), 128, 0, st>>>(keys.as<unsigned long long>(), rstart.as<int64_t>(), n_nodes,
                                                       c->row_ptr.as<int32_t>(), c->col.as<int32_t>(),
                                                       c->slot_ptr.as<int32_t>(), c->diag_slot.as<int32_t>(),
                                                       c->entries.as<uint32_t>());
    ECT_CHECK_LAUNCH();
    c->h_row_ptr = hrp;
    c->h_col.resize(nnzb);
    ECT_CUDA(cudaMemcpyAsync(c->h_col.data(), c->col.p, sizeof(int32_t) * nnzb, cudaMemcpyDeviceToHost, st));
    ECT_CUDA(cudaStreamSynchronize(st));
    c->mesh_set = true;
}
