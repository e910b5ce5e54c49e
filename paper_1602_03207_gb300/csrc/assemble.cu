// Kernel (a): race-free P1 assembly of the A-V system into 4x4 complex blocks.
//
// For tet K with volume |K| and barycentric gradients g_a, the coupled form
// of Sec. 2 (L11 + L12 + L21 + L22 after the V equation is scaled by
// -1/(i omega), with the -i omega sigma mass term inside L11 and the gauge
// penalty delta sigma V of Sec. 4 inside L22) gives the node-pair block
// (test node a, trial node b), rows/cols ordered (A_x, A_y, A_z, V):
//   AA_pq = |K| [nu (d_pq g_a.g_b - g_aq g_bp) + nu_t g_ap g_bq]
//           - i omega sigma |K| (1 + d_ab)/20 d_pq
//   AV_p  = -sigma |K| g_bp / 4,        VA_q = -sigma |K| g_aq / 4
//   VV    = -(sigma/(i omega)) |K| (g_a.g_b + delta (1 + d_ab)/20)
// One thread owns one block and sums the contributions of every tet that
// shares its node pair (the list built in mesh_setup.cu), so no two threads
// write the same value and the summation order is fixed.  The constraints
// follow: A.n = 0 by elimination (zero row and column, unit diagonal) and
// the identity on V at nodes that touch no conducting tet.  A configuration
// with the impedance boundary condition (ibc.cu) skips its plate tets and
// adds the surface term of each plate face to the blocks of its node pairs
// (again one thread per block, fixed order).  Finally the
// symmetric scaling S = T M T with T = diag(|M_ii|^-1/2) is formed in FP64
// and, on request, rounded to an FP32 copy.
#include <cmath>

#include "common.cuh"

namespace {

__device__ __forceinline__ int row_of_slot(const int32_t* __restrict__ row_ptr, int64_t n_rows, int slot) {
    int lo = 0, hi = (int)n_rows - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (row_ptr[mid] <= slot) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(128) k_assemble(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col, const int32_t* __restrict__ slot_ptr,
    const uint32_t* __restrict__ entries, const double* __restrict__ geo, const double* __restrict__ sigma,
    const double* __restrict__ nu, const uint8_t* __restrict__ fixmask, int64_t n_rows, int64_t nnzb,
    double nu_t, double omega, double delta, const uint8_t* __restrict__ tvoid, const int32_t* __restrict__ s_ptr,
    const uint32_t* __restrict__ s_ent, const double* __restrict__ s_geo, double2 s_coef,
    double2* __restrict__ val) {
    int64_t slot = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (slot >= nnzb) return;
    double re[16], im[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) re[e] = im[e] = 0.0;
    const double inv_omega = 1.0 / omega;
    for (int32_t q = slot_ptr[slot]; q < slot_ptr[slot + 1]; ++q) {
        uint32_t ent = entries[q];
        int64_t t = ent >> 4;
        if (tvoid && tvoid[t]) continue;  // plate removed by the impedance boundary condition
        int a = (ent >> 2) & 3, b = ent & 3;
        const double* g = geo + 16 * t;
        double vol = g[0];
        double ga[3] = {g[1 + 3 * a], g[2 + 3 * a], g[3 + 3 * a]};
        double gb[3] = {g[1 + 3 * b], g[2 + 3 * b], g[3 + 3 * b]};
        double s = sigma[t], n = nu[t];
        double gab = ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2];
        double mass = (a == b ? 2.0 : 1.0) / 20.0;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                double cc = (p == r ? gab : 0.0) - ga[r] * gb[p];
                re[4 * p + r] += vol * (n * cc + nu_t * ga[p] * gb[r]);
            }
            im[5 * p] -= omega * s * vol * mass;
            re[4 * p + 3] -= 0.25 * s * vol * gb[p];
            re[12 + p] -= 0.25 * s * vol * ga[p];
        }
        im[15] += s * inv_omega * vol * (gab + delta * mass);
    }
    if (s_ptr) {
        // impedance condition on the plate surface: s_coef |F| (1 + d_ab)/12 (d_ij - n_i n_j)
        for (int32_t q = s_ptr[slot]; q < s_ptr[slot + 1]; ++q) {
            const uint32_t ent = s_ent[q];
            const double* fg = s_geo + 4 * (int64_t)(ent >> 4);
            const int a = (ent >> 2) & 3, b = ent & 3;
            const double m = fg[0] * (a == b ? 2.0 : 1.0) / 12.0;
            const double nn[3] = {fg[1], fg[2], fg[3]};
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    const double pr = m * ((p == r ? 1.0 : 0.0) - nn[p] * nn[r]);
                    re[4 * p + r] += s_coef.x * pr;
                    im[4 * p + r] += s_coef.y * pr;
                }
        }
    }
    int row = row_of_slot(row_ptr, n_rows, (int)slot);
    int cl = col[slot];
    unsigned fr = fixmask[row], fc = fixmask[cl];
    double2* out = val + 16 * slot;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            double2 v = make_double2(re[4 * p + r], im[4 * p + r]);
            if (((fr >> p) & 1u) || ((fc >> r) & 1u)) v = make_double2(0.0, 0.0);
            if (row == cl && p == r && ((fr >> p) & 1u)) v = make_double2(1.0, 0.0);
            out[4 * p + r] = v;
        }
    }
}

// Frequency sweep: the values of one configuration at F frequencies in one
// pass over the pattern.  Only three parts of a block depend on omega: the
// A-A mass term (-i omega sigma |K| (1 + d_ab)/20 on the diagonal of the
// component block), the V-V term (+i (sigma/omega) |K| (g_a.g_b + delta
// (1 + d_ab)/20)) and the surface term of an impedance boundary condition
// (coefficient ~ sqrt(omega)); the thread sums the omega-free parts once and
// writes F blocks.
constexpr int MAX_SWEEP = 16;
struct SweepOut {
    double omega[MAX_SWEEP];
    double2 s_coef[MAX_SWEEP];
    double2* val[MAX_SWEEP];
    int F;
};

__global__ void __launch_bounds__(128) k_assemble_sweep(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col, const int32_t* __restrict__ slot_ptr,
    const uint32_t* __restrict__ entries, const double* __restrict__ geo, const double* __restrict__ sigma,
    const double* __restrict__ nu, const uint8_t* __restrict__ fixmask, int64_t n_rows, int64_t nnzb, double nu_t,
    double delta, const uint8_t* __restrict__ tvoid, const int32_t* __restrict__ s_ptr,
    const uint32_t* __restrict__ s_ent, const double* __restrict__ s_geo, const SweepOut out) {
    int64_t slot = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (slot >= nnzb) return;
    double re[16], sp[9];
    double mass_aa = 0.0, vv = 0.0;  // sum sigma |K| (1 + d_ab)/20 and sum sigma |K| (g_a.g_b + delta (1 + d_ab)/20)
#pragma unroll
    for (int e = 0; e < 16; ++e) re[e] = 0.0;
#pragma unroll
    for (int e = 0; e < 9; ++e) sp[e] = 0.0;
    for (int32_t q = slot_ptr[slot]; q < slot_ptr[slot + 1]; ++q) {
        uint32_t ent = entries[q];
        int64_t t = ent >> 4;
        if (tvoid && tvoid[t]) continue;
        int a = (ent >> 2) & 3, b = ent & 3;
        const double* g = geo + 16 * t;
        double vol = g[0];
        double ga[3] = {g[1 + 3 * a], g[2 + 3 * a], g[3 + 3 * a]};
        double gb[3] = {g[1 + 3 * b], g[2 + 3 * b], g[3 + 3 * b]};
        double s = sigma[t], n = nu[t];
        double gab = ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2];
        double mass = (a == b ? 2.0 : 1.0) / 20.0;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                double cc = (p == r ? gab : 0.0) - ga[r] * gb[p];
                re[4 * p + r] += vol * (n * cc + nu_t * ga[p] * gb[r]);
            }
            re[4 * p + 3] -= 0.25 * s * vol * gb[p];
            re[12 + p] -= 0.25 * s * vol * ga[p];
        }
        mass_aa += s * vol * mass;
        vv += s * vol * (gab + delta * mass);
    }
    if (s_ptr) {
        for (int32_t q = s_ptr[slot]; q < s_ptr[slot + 1]; ++q) {
            const uint32_t ent = s_ent[q];
            const double* fg = s_geo + 4 * (int64_t)(ent >> 4);
            const int a = (ent >> 2) & 3, b = ent & 3;
            const double m = fg[0] * (a == b ? 2.0 : 1.0) / 12.0;
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int r = 0; r < 3; ++r) sp[3 * p + r] += m * ((p == r ? 1.0 : 0.0) - fg[1 + p] * fg[1 + r]);
        }
    }
    int row = row_of_slot(row_ptr, n_rows, (int)slot);
    int cl = col[slot];
    unsigned fr = fixmask[row], fc = fixmask[cl];
    for (int f = 0; f < out.F; ++f) {
        const double om = out.omega[f];
        const double2 sc = out.s_coef[f];
        double2* o = out.val[f] + 16 * slot;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                double vr = re[4 * p + r], vi = 0.0;
                if (p < 3 && r < 3) {
                    if (p == r) vi -= om * mass_aa;
                    vr += sc.x * sp[3 * p + r];
                    vi += sc.y * sp[3 * p + r];
                }
                if (p == 3 && r == 3) vi += vv / om;
                double2 v = make_double2(vr, vi);
                if (((fr >> p) & 1u) || ((fc >> r) & 1u)) v = make_double2(0.0, 0.0);
                if (row == cl && p == r && ((fr >> p) & 1u)) v = make_double2(1.0, 0.0);
                o[4 * p + r] = v;
            }
        }
    }
}

__global__ void k_scaling(const double2* __restrict__ val, const int32_t* __restrict__ diag_slot, int64_t n_rows,
                          double* __restrict__ t) {
    int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (d >= 4 * n_rows) return;
    int64_t row = d >> 2;
    int p = (int)(d & 3);
    double2 m = val[16 * (int64_t)diag_slot[row] + 5 * p];
    double a = sqrt(m.x * m.x + m.y * m.y);
    t[d] = a > 0.0 ? 1.0 / sqrt(a) : 1.0;
}

__global__ void k_scale_matrix(const double2* __restrict__ val, const int32_t* __restrict__ row_ptr,
                               const int32_t* __restrict__ col, const double* __restrict__ t, int64_t n_rows,
                               int64_t nnzb, double2* __restrict__ sval, float2* __restrict__ sval32,
                               float2* __restrict__ sval32lo, float* __restrict__ sval32p) {
    int64_t slot = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (slot >= nnzb) return;
    int row = row_of_slot(row_ptr, n_rows, (int)slot);
    int cl = col[slot];
    double tr[4], tc[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        tr[p] = t[4 * (int64_t)row + p];
        tc[p] = t[4 * (int64_t)cl + p];
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            double2 m = val[16 * slot + 4 * p + r];
            double s = tr[p] * tc[r];
            double2 v = make_double2(m.x * s, m.y * s);
            sval[16 * slot + 4 * p + r] = v;
            if (sval32) {
                const float2 h = make_float2((float)v.x, (float)v.y);
                sval32[16 * slot + 4 * p + r] = h;
                float* q = sval32p + 32 * slot + 16 * (p >> 1) + 4 * r + (p & 1);  // row-pair layout
                q[0] = h.x;
                q[2] = h.y;
                sval32lo[16 * slot + 4 * p + r] =
                    make_float2((float)(v.x - (double)h.x), (float)(v.y - (double)h.y));
            }
        }
}

// -(i omega / Z) with Z = (1 - i)/(delta sigma_p), delta = sqrt(2 nu_p / (omega sigma_p)):
// (omega delta sigma_p / 2)(1 - i)
double2 ibc_coefficient_at(double omega, const Matrix& M) {
    if (!M.ibc) return make_double2(0.0, 0.0);
    const double delta = std::sqrt(2.0 * M.ibc_nu / (omega * M.ibc_sigma));
    const double a = 0.5 * omega * delta * M.ibc_sigma;
    return make_double2(a, -a);
}
double2 ibc_coefficient(const ect_ctx* c, const Matrix& M) { return ibc_coefficient_at(c->omega, M); }

// the scaling t and the scaled copies of an assembled matrix
void scale_matrix(ect_ctx* c, Matrix& M, bool f32) {
    cudaStream_t st = c->stream;
    const int64_t nnzb = c->nnzb, N = c->n_nodes;
    k_scaling<<<grid_for(4 * N, 256), 256, 0, st>>>(M.val.as<double2>(), c->diag_slot.as<int32_t>(), N,
                                                    M.t.as<double>());
    ECT_CHECK_LAUNCH();
    k_scale_matrix<<<grid_for(nnzb, 128), 128, 0, st>>>(M.val.as<double2>(), c->row_ptr.as<int32_t>(),
                                                        c->col.as<int32_t>(), M.t.as<double>(), N, nnzb,
                                                        M.sval.as<double2>(), f32 ? M.sval32.as<float2>() : nullptr,
                                                        f32 ? M.sval32lo.as<float2>() : nullptr,
                                                        f32 ? M.sval32p.as<float>() : nullptr);
    ECT_CHECK_LAUNCH();
    ++M.val_gen;
}

void alloc_values(ect_ctx* c, Matrix& M, bool f32) {
    const int64_t nnzb = c->nnzb, N = c->n_nodes;
    M.val.alloc(sizeof(double2) * 16 * nnzb);
    M.sval.alloc(sizeof(double2) * 16 * nnzb);
    M.t.alloc(sizeof(double) * 4 * N);
    if (f32) {
        M.sval32.alloc(sizeof(float2) * 16 * nnzb);
        M.sval32lo.alloc(sizeof(float2) * 16 * nnzb);
        M.sval32p.alloc(sizeof(float2) * 16 * nnzb);
    } else {
        M.sval32.release();
        M.sval32lo.release();
        M.sval32p.release();
    }
    M.sval32t.release();  // rebuilt from sval32 on demand
    M.t_gen = 0;
}

}  // namespace

void assemble_matrix(ect_ctx* c, int which, int precision_mask) {
    ECT_REQUIRE(c->mesh_set, ECT_ERR_STATE, "ect_set_mesh must come before ect_assemble");
    ECT_REQUIRE(c->physics_set, ECT_ERR_STATE, "ect_set_physics must come before ect_assemble");
    ECT_REQUIRE(which == ECT_VACUUM || which == ECT_DEFECT, ECT_ERR_ARG, "which must be ECT_VACUUM or ECT_DEFECT");
    ECT_REQUIRE((precision_mask & ~(ECT_F64 | ECT_F32)) == 0, ECT_ERR_ARG, "bad precision mask");
    Matrix& M = c->mat[which];
    cudaStream_t st = c->stream;
    const int64_t nnzb = c->nnzb, N = c->n_nodes;
    bool f32 = (precision_mask & ECT_F32) != 0;
    alloc_values(c, M, f32);
    k_assemble<<<grid_for(nnzb, 128), 128, 0, st>>>(
        c->row_ptr.as<int32_t>(), c->col.as<int32_t>(), c->slot_ptr.as<int32_t>(), c->entries.as<uint32_t>(),
        c->geo.as<double>(), M.sigma.as<double>(), M.nu.as<double>(), M.fixmask.as<uint8_t>(), N, nnzb,
        c->nu_tilde, c->omega, c->delta, M.ibc ? M.tvoid.as<uint8_t>() : nullptr,
        M.ibc ? M.s_ptr.as<int32_t>() : nullptr, M.ibc ? M.s_ent.as<uint32_t>() : nullptr,
        M.ibc ? M.s_geo.as<double>() : nullptr, ibc_coefficient(c, M), M.val.as<double2>());
    ECT_CHECK_LAUNCH();
    scale_matrix(c, M, f32);
    M.assembled = true;
    M.has_f32 = f32;
    M.omega = c->omega;
    M.pc_f64 = M.pc_f32 = false;
}

// Frequency sweep: both configurations at F frequencies (matrices 2 + 2 f + c),
// sharing the pattern, the per-tet coefficients, the constraint mask and an
// impedance boundary condition of the context's configuration c.  One
// k_assemble_sweep launch per configuration writes its F value sets.
void assemble_sweep(ect_ctx* c, const double* freq_hz, int n_freq, int precision_mask) {
    ECT_REQUIRE(c->mesh_set, ECT_ERR_STATE, "ect_set_mesh must come before ect_assemble_sweep");
    ECT_REQUIRE(c->physics_set, ECT_ERR_STATE, "ect_set_physics must come before ect_assemble_sweep");
    ECT_REQUIRE(freq_hz && n_freq >= 1 && n_freq <= MAX_SWEEP, ECT_ERR_ARG, "need 1 to 16 frequencies");
    ECT_REQUIRE((precision_mask & ~(ECT_F64 | ECT_F32)) == 0, ECT_ERR_ARG, "bad precision mask");
    for (int f = 0; f < n_freq; ++f)
        ECT_REQUIRE(std::isfinite(freq_hz[f]) && freq_hz[f] > 0.0, ECT_ERR_ARG, "frequencies must be > 0");
    workspace_free(c);
    c->smat.clear();
    c->sweep_omega.clear();
    for (int f = 0; f < n_freq; ++f) c->sweep_omega.push_back(2.0 * 3.14159265358979323846 * freq_hz[f]);
    const bool f32 = (precision_mask & ECT_F32) != 0;
    cudaStream_t st = c->stream;
    const int64_t nnzb = c->nnzb, N = c->n_nodes;
    for (int f = 0; f < n_freq; ++f)
        for (int cfg = 0; cfg < 2; ++cfg) {
            c->smat.emplace_back();
            Matrix& M = c->smat.back();
            const Matrix& B = c->mat[cfg];
            M.h_cond = B.h_cond;
            M.h_fix = B.h_fix;
            M.ibc = B.ibc;
            M.ibc_sigma = B.ibc_sigma;
            M.ibc_nu = B.ibc_nu;
            M.fixmask.alloc(N);
            ECT_CUDA(cudaMemcpyAsync(M.fixmask.p, B.fixmask.p, N, cudaMemcpyDeviceToDevice, st));
            alloc_values(c, M, f32);
        }
    for (int cfg = 0; cfg < 2; ++cfg) {
        const Matrix& B = c->mat[cfg];
        SweepOut out;
        out.F = n_freq;
        for (int f = 0; f < n_freq; ++f) {
            out.omega[f] = c->sweep_omega[f];
            out.s_coef[f] = ibc_coefficient_at(c->sweep_omega[f], B);
            out.val[f] = c->smat[2 * f + cfg].val.as<double2>();
        }
        k_assemble_sweep<<<grid_for(nnzb, 128), 128, 0, st>>>(
            c->row_ptr.as<int32_t>(), c->col.as<int32_t>(), c->slot_ptr.as<int32_t>(), c->entries.as<uint32_t>(),
            c->geo.as<double>(), B.sigma.as<double>(), B.nu.as<double>(), B.fixmask.as<uint8_t>(), N, nnzb,
            c->nu_tilde, c->delta, B.ibc ? B.tvoid.as<uint8_t>() : nullptr, B.ibc ? B.s_ptr.as<int32_t>() : nullptr,
            B.ibc ? B.s_ent.as<uint32_t>() : nullptr, B.ibc ? B.s_geo.as<double>() : nullptr, out);
        ECT_CHECK_LAUNCH();
        for (int f = 0; f < n_freq; ++f) {
            Matrix& M = c->smat[2 * f + cfg];
            scale_matrix(c, M, f32);
            M.assembled = true;
            M.has_f32 = f32;
            M.omega = c->sweep_omega[f];
        }
    }
    ECT_CUDA(cudaStreamSynchronize(st));
}
