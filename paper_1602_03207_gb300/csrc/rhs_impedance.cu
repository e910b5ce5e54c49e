// Coil source term (Step 6 of Sec. 3) and kernel (e), the Delta Z reduction.
//
// Source: the paper builds the load as the mass matrix times the
// interpolated analytic source J = J_e (-y, x, 0)/sqrt(x^2 + y^2) (Sec. 3-4).
// Here the mass matrix is taken over the coil tets only, each weighted by the
// fraction f_K of 35 interior sample points (barycentric weights
// (4 n_a + 1)/20, n0 + n1 + n2 + n3 = 4) inside the coil annulus:
//   b_(a,i) = sum_{K containing a} f_K |K|/20 (J_i(x_a) + sum_{b in K} J_i(x_b)).
// The point-in-coil decisions are made with every operation rounded
// separately (no fused multiply-add), so they are reproducible bit for bit.
// Kernel 1 counts the points per (position, tet) with a cheap z-range
// rejection; kernel 2 gathers, per (position, node), over the tets that
// contain the node (the diagonal block's contribution list), so no atomics.
//
// Delta Z (Eq. impedkl read as the discrete reciprocity identity):
//   dZ_kl = (i omega/(I_k I_l)) sum_{K in Omega_d} u_k^0|_K^T (E_K^d - E_K^0) u_l^d|_K,
// with E_K the element matrix of kernel (a); the difference is linear in
// (sigma_d - sigma_0, nu_d - nu_0) and the nu_tilde term cancels.  One thread
// per defect tet evaluates the four (k, l) bilinear forms; per-CTA partial
// sums are added in a fixed order on the host.  The coil-EMF difference
// -(i omega/(I_k I_l)) b_k^T (u_l^d - u_l^0) is reduced alongside as a check.
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace {

__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }

__global__ void k_coil_counts(const double* __restrict__ xyz, const int32_t* __restrict__ tets, int64_t n_tets,
                              double r_in, double r_out, double length, double z_off, const double* __restrict__ zp,
                              uint8_t* __restrict__ cnt) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int pos = blockIdx.y;
    if (t >= n_tets) return;
    double p[4][3];
    double zmin = 1e300, zmax = -1e300, r2max = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int n = tets[4 * t + a];
#pragma unroll
        for (int i = 0; i < 3; ++i) p[a][i] = xyz[3 * (int64_t)n + i];
        zmin = fmin(zmin, p[a][2]);
        zmax = fmax(zmax, p[a][2]);
        r2max = fmax(r2max, p[a][0] * p[a][0] + p[a][1] * p[a][1]);
    }
    const double zc = rn_add(zp[pos], z_off);
    const double half = rn_mul(0.5, length);
    const double margin = 1e-9;
    uint8_t count = 0;
    if (!(zmax < zc - half - margin || zmin > zc + half + margin || r2max < r_in * r_in * (1.0 - 1e-9))) {
        const double ri2 = rn_mul(r_in, r_in), ro2 = rn_mul(r_out, r_out);
        for (int n0 = 0; n0 <= 4; ++n0)
            for (int n1 = 0; n1 <= 4 - n0; ++n1)
                for (int n2 = 0; n2 <= 4 - n0 - n1; ++n2) {
                    const int n3 = 4 - n0 - n1 - n2;
                    const double m[4] = {4.0 * n0 + 1.0, 4.0 * n1 + 1.0, 4.0 * n2 + 1.0, 4.0 * n3 + 1.0};
                    double q[3];
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        double acc = rn_mul(m[0], p[0][i]);
                        acc = rn_add(acc, rn_mul(m[1], p[1][i]));
                        acc = rn_add(acc, rn_mul(m[2], p[2][i]));
                        acc = rn_add(acc, rn_mul(m[3], p[3][i]));
                        q[i] = rn_mul(acc, 0.05);
                    }
                    const double r2 = rn_add(rn_mul(q[0], q[0]), rn_mul(q[1], q[1]));
                    const double dz = fabs(__dsub_rn(q[2], zc));
                    if (r2 >= ri2 && r2 <= ro2 && dz <= half) ++count;
                }
    }
    cnt[(int64_t)pos * n_tets + t] = count;
}

__device__ __forceinline__ void source_at(const double* __restrict__ xyz, int n, double J_e, double& jx, double& jy) {
    const double x = xyz[3 * (int64_t)n], y = xyz[3 * (int64_t)n + 1];
    const double r = sqrt(x * x + y * y);
    if (r < 1e-12) {
        jx = jy = 0.0;
        return;
    }
    jx = -J_e * y / r;
    jy = J_e * x / r;
}

__global__ void k_coil_gather(const double* __restrict__ xyz, const int32_t* __restrict__ tets,
                              const double* __restrict__ geo, const int32_t* __restrict__ diag_slot,
                              const int32_t* __restrict__ slot_ptr, const uint32_t* __restrict__ entries,
                              const uint8_t* __restrict__ cnt, const uint8_t* __restrict__ bc, int64_t n_nodes,
                              int64_t n_tets, double J_e, double2* __restrict__ out, int64_t pos_stride) {
    const int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int pos = blockIdx.y;
    if (node >= n_nodes) return;
    const int s = diag_slot[node];
    double bx = 0.0, by = 0.0;
    for (int32_t q = slot_ptr[s]; q < slot_ptr[s + 1]; ++q) {
        const uint32_t ent = entries[q];
        const int64_t t = ent >> 4;
        const int a = (ent >> 2) & 3;
        const uint8_t c = cnt[(int64_t)pos * n_tets + t];
        if (!c) continue;
        const double f = (double)c / 35.0;
        const double w = f * geo[16 * t] / 20.0;
        double sx = 0.0, sy = 0.0, ax = 0.0, ay = 0.0;
        for (int b = 0; b < 4; ++b) {
            double jx, jy;
            source_at(xyz, tets[4 * t + b], J_e, jx, jy);
            sx += jx;
            sy += jy;
            if (b == a) {
                ax = jx;
                ay = jy;
            }
        }
        bx += w * (ax + sx);
        by += w * (ay + sy);
    }
    const uint8_t m = bc[node];
    double2* o = out + (int64_t)pos * pos_stride + 4 * node;
    o[0] = make_double2((m & 1) ? 0.0 : bx, 0.0);
    o[1] = make_double2((m & 2) ? 0.0 : by, 0.0);
    o[2] = make_double2(0.0, 0.0);
    o[3] = make_double2(0.0, 0.0);
}

// per defect tet, the four bilinear forms u0_k^T (E_d - E_0) ud_l
constexpr int DZ_TPB = 128;

__global__ void __launch_bounds__(DZ_TPB) k_delta_z(const int32_t* __restrict__ omega_d, int64_t n_d,
                                                    const int32_t* __restrict__ tets, const double* __restrict__ geo,
                                                    const double* __restrict__ s0, const double* __restrict__ n0,
                                                    const double* __restrict__ s1, const double* __restrict__ n1,
                                                    double omega, double delta, const double2* __restrict__ u0,
                                                    const double2* __restrict__ ud, int64_t nvec,
                                                    double* __restrict__ part) {
    __shared__ double sh[8 * 8];
    const int pos = blockIdx.y;
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    const double2* U0 = u0 + (int64_t)pos * 2 * nvec;
    const double2* Ud = ud + (int64_t)pos * 2 * nvec;
    for (int64_t i = blockIdx.x * (int64_t)DZ_TPB + threadIdx.x; i < n_d; i += (int64_t)gridDim.x * DZ_TPB) {
        const int64_t t = omega_d[i];
        const double* g = geo + 16 * t;
        const double vol = g[0];
        const double ds = s1[t] - s0[t], dn = n1[t] - n0[t];
        int nd[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) nd[a] = tets[4 * t + a];
        // w_l[b][q] = sum over b, q of D[a,b][p][q] ud_l[b][q] accumulated into y_l[a][p]
        double2 y[2][4][4];
#pragma unroll
        for (int l = 0; l < 2; ++l)
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int p = 0; p < 4; ++p) y[l][a][p] = make_double2(0.0, 0.0);
        for (int a = 0; a < 4; ++a) {
            const double ga[3] = {g[1 + 3 * a], g[2 + 3 * a], g[3 + 3 * a]};
            for (int b = 0; b < 4; ++b) {
                const double gb[3] = {g[1 + 3 * b], g[2 + 3 * b], g[3 + 3 * b]};
                const double gab = ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2];
                const double mass = (a == b ? 2.0 : 1.0) / 20.0;
                double re[16], im[16];
#pragma unroll
                for (int p = 0; p < 3; ++p) {
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        const double cc = (p == r ? gab : 0.0) - ga[r] * gb[p];
                        re[4 * p + r] = vol * dn * cc;
                        im[4 * p + r] = (p == r) ? -omega * ds * vol * mass : 0.0;
                    }
                    re[4 * p + 3] = -0.25 * ds * vol * gb[p];
                    im[4 * p + 3] = 0.0;
                    re[12 + p] = -0.25 * ds * vol * ga[p];
                    im[12 + p] = 0.0;
                }
                re[15] = 0.0;
                im[15] = ds / omega * vol * (gab + delta * mass);
                for (int l = 0; l < 2; ++l) {
                    const double2* ub = Ud + (int64_t)l * nvec + 4 * (int64_t)nd[b];
                    const double2 u[4] = {ub[0], ub[1], ub[2], ub[3]};
#pragma unroll
                    for (int p = 0; p < 4; ++p)
#pragma unroll
                        for (int r = 0; r < 4; ++r) cfma(y[l][a][p], make_double2(re[4 * p + r], im[4 * p + r]), u[r]);
                }
            }
        }
        for (int kk = 0; kk < 2; ++kk)
            for (int a = 0; a < 4; ++a) {
                const double2* ua = U0 + (int64_t)kk * nvec + 4 * (int64_t)nd[a];
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const double2 v = ua[p];
#pragma unroll
                    for (int l = 0; l < 2; ++l) {
                        const double2 pr = cmul(v, y[l][a][p]);
                        acc[2 * (2 * kk + l)] += pr.x;
                        acc[2 * (2 * kk + l) + 1] += pr.y;
                    }
                }
            }
    }
    // block reduce 8 doubles
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = warp_sum(acc[q]);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 8; ++q) sh[warp * 8 + q] = acc[q];
    __syncthreads();
    if (threadIdx.x < 8) {
        double s = 0.0;
        for (int w = 0; w < DZ_TPB / 32; ++w) s += sh[w * 8 + threadIdx.x];
        part[((int64_t)pos * gridDim.x + blockIdx.x) * 8 + threadIdx.x] = s;
    }
}

// b_k^T (ud_l - u0_l) partials (bilinear)
__global__ void __launch_bounds__(256) k_emf(const double2* __restrict__ b, const double2* __restrict__ u0,
                                             const double2* __restrict__ ud, int64_t nvec, double* __restrict__ part) {
    __shared__ double sh[8 * 8];
    const int pos = blockIdx.y;
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    const double2* B = b + (int64_t)pos * 2 * nvec;
    const double2* U0 = u0 + (int64_t)pos * 2 * nvec;
    const double2* Ud = ud + (int64_t)pos * 2 * nvec;
    for (int64_t e = blockIdx.x * 256ll + threadIdx.x; e < nvec; e += (int64_t)gridDim.x * 256) {
        const double2 bk[2] = {B[e], B[nvec + e]};
        const double2 du[2] = {csub(Ud[e], U0[e]), csub(Ud[nvec + e], U0[nvec + e])};
#pragma unroll
        for (int kk = 0; kk < 2; ++kk)
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                const double2 pr = cmul(bk[kk], du[l]);
                acc[2 * (2 * kk + l)] += pr.x;
                acc[2 * (2 * kk + l) + 1] += pr.y;
            }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = warp_sum(acc[q]);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 8; ++q) sh[warp * 8 + q] = acc[q];
    __syncthreads();
    if (threadIdx.x < 8) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += sh[w * 8 + threadIdx.x];
        part[((int64_t)pos * gridDim.x + blockIdx.x) * 8 + threadIdx.x] = s;
    }
}

}  // namespace

void coil_rhs(ect_ctx* c, const ect_coil& coil, const double* h_z, int k, double2* d_rhs) {
    ECT_REQUIRE(c->mesh_set, ECT_ERR_STATE, "ect_set_mesh must come first");
    ECT_REQUIRE(h_z && d_rhs && k >= 1 && k <= 65535, ECT_ERR_ARG, "bad coil_rhs arguments");
    ECT_REQUIRE(coil.r_in >= 0.0 && coil.r_out > coil.r_in && coil.length > 0.0, ECT_ERR_ARG, "bad coil geometry");
    cudaStream_t st = c->stream;
    const int64_t T = c->n_tets, N = c->n_nodes;
    DevBuf zp, cnt;
    zp.alloc(sizeof(double) * k);
    cnt.alloc((size_t)k * T);
    ECT_CUDA(cudaMemcpyAsync(zp.p, h_z, sizeof(double) * k, cudaMemcpyHostToDevice, st));
    k_coil_counts<<<dim3(grid_for(T, 128), k), 128, 0, st>>>(c->xyz.as<double>(), c->tets.as<int32_t>(), T, coil.r_in,
                                                              coil.r_out, coil.length, coil.z_offset, zp.as<double>(),
                                                              cnt.as<uint8_t>());
    ECT_CHECK_LAUNCH();
    k_coil_gather<<<dim3(grid_for(N, 128), k), 128, 0, st>>>(
        c->xyz.as<double>(), c->tets.as<int32_t>(), c->geo.as<double>(), c->diag_slot.as<int32_t>(),
        c->slot_ptr.as<int32_t>(), c->entries.as<uint32_t>(), cnt.as<uint8_t>(), c->bc.as<uint8_t>(), N, T, coil.J_e,
        d_rhs, 4 * N);
    ECT_CHECK_LAUNCH();
    ECT_CUDA(cudaStreamSynchronize(st));
}

// u0, ud, b: [n_pos][2][4N]; h_dz (and h_dz_emf): [n_pos][2][2] complex
void delta_z(ect_ctx* c, const double2* u0, const double2* ud, const double2* b, const double* cur, int n_pos,
             double* h_dz, double* h_dz_emf, double omega) {
    if (omega <= 0.0) omega = c->omega;
    ECT_REQUIRE(c->mesh_set && c->physics_set, ECT_ERR_STATE, "mesh and physics must be set");
    ECT_REQUIRE(u0 && ud && cur && h_dz && n_pos >= 1, ECT_ERR_ARG, "bad delta_z arguments");
    ECT_REQUIRE(cur[0] != 0.0 && cur[1] != 0.0, ECT_ERR_ARG, "coil currents must be non-zero");
    ECT_REQUIRE(!h_dz_emf || b, ECT_ERR_ARG, "h_dz_emf needs d_b");
    // With the impedance boundary condition the plate's volume fields are not computed, so
    // the volume form of Eq. impedkl has nothing to integrate: Delta Z is the coil-EMF
    // difference, which needs the sources.
    const bool emf_only = c->mat[0].ibc || c->mat[1].ibc;
    ECT_REQUIRE(!emf_only || b, ECT_ERR_ARG, "with the impedance boundary condition Delta Z needs d_b (EMF form)");
    std::vector<double> emf_tmp;
    if (emf_only && !h_dz_emf) {
        emf_tmp.resize(8 * (size_t)n_pos);
        h_dz_emf = emf_tmp.data();
    }
    cudaStream_t st = c->stream;
    const int64_t nvec = 4 * c->n_nodes;
    int G = (int)std::min<int64_t>(std::max<int64_t>(1, (c->n_omega_d + DZ_TPB - 1) / DZ_TPB), 304);
    int Ge = (int)std::min<int64_t>((nvec + 255) / 256, 304);
    DevBuf part, parte;
    part.alloc(sizeof(double) * 8 * G * n_pos);
    parte.alloc(sizeof(double) * 8 * Ge * n_pos);
    k_delta_z<<<dim3(G, n_pos), DZ_TPB, 0, st>>>(c->omega_d.as<int32_t>(), c->n_omega_d, c->tets.as<int32_t>(),
                                                 c->geo.as<double>(), c->mat[0].sigma.as<double>(),
                                                 c->mat[0].nu.as<double>(), c->mat[1].sigma.as<double>(),
                                                 c->mat[1].nu.as<double>(), omega, c->delta, u0, ud, nvec,
                                                 part.as<double>());
    ECT_CHECK_LAUNCH();
    if (h_dz_emf && b) {
        k_emf<<<dim3(Ge, n_pos), 256, 0, st>>>(b, u0, ud, nvec, parte.as<double>());
        ECT_CHECK_LAUNCH();
    }
    std::vector<double> hp(8 * G * n_pos), he(8 * Ge * n_pos);
    ECT_CUDA(cudaMemcpyAsync(hp.data(), part.p, part.bytes, cudaMemcpyDeviceToHost, st));
    if (h_dz_emf && b) ECT_CUDA(cudaMemcpyAsync(he.data(), parte.p, parte.bytes, cudaMemcpyDeviceToHost, st));
    ECT_CUDA(cudaStreamSynchronize(st));
    const double om = omega;
    for (int p = 0; p < n_pos; ++p) {
        for (int kl = 0; kl < 4; ++kl) {
            const int kk = kl >> 1, l = kl & 1;
            double sr = 0.0, si = 0.0;
            for (int g = 0; g < G; ++g) {
                sr += hp[((int64_t)p * G + g) * 8 + 2 * kl];
                si += hp[((int64_t)p * G + g) * 8 + 2 * kl + 1];
            }
            // (i omega / (I_k I_l)) * (sr + i si)
            const double f = om / (cur[kk] * cur[l]);
            h_dz[(int64_t)p * 8 + 2 * kl] = -f * si;
            h_dz[(int64_t)p * 8 + 2 * kl + 1] = f * sr;
            if (h_dz_emf && b) {
                double er = 0.0, ei = 0.0;
                for (int g = 0; g < Ge; ++g) {
                    er += he[((int64_t)p * Ge + g) * 8 + 2 * kl];
                    ei += he[((int64_t)p * Ge + g) * 8 + 2 * kl + 1];
                }
                // -(i omega / (I_k I_l)) * (er + i ei)
                h_dz_emf[(int64_t)p * 8 + 2 * kl] = f * ei;
                h_dz_emf[(int64_t)p * 8 + 2 * kl + 1] = -f * er;
            }
        }
    }
    if (emf_only)
        for (int64_t e = 0; e < 8 * (int64_t)n_pos; ++e) h_dz[e] = h_dz_emf[e];
}

// ----------------------------------------------------------------------------
// Delta Z without any device allocation.
//
// Some callers cannot call cudaMalloc: an application whose device memory is
// entirely owned by its own pool allocator, or a caller that must not hit the
// allocator's latency or device synchronisation (cudaFree synchronises the
// device) in the middle of its own stream work.  ect_delta_z_static serves
// them: its scratch (per-CTA partial sums and the reduced results) lives in
// the file-scope device array below, sized for at most DZ_STATIC_MAX_POS
// positions per call, which every GPU that loads the library keeps until the
// process exits.  Every call reuses the same array, so calls that overlap on
// the GPU race; each call overwrites everything it reads, so nothing has to
// start at zero.
// ----------------------------------------------------------------------------
namespace {

constexpr int DZ_STATIC_MAX_POS = 64;
constexpr int DZ_STATIC_G = 256;     // CTAs of the Delta Z kernel per position
constexpr int DZ_STATIC_GE = 256;    // CTAs of the EMF kernel per position
constexpr int64_t DZ_STATIC_PART = (int64_t)DZ_STATIC_MAX_POS * (DZ_STATIC_G + DZ_STATIC_GE) * 8;
constexpr int64_t DZ_STATIC_DOUBLES = DZ_STATIC_PART + (int64_t)DZ_STATIC_MAX_POS * 16;  // 2.1 MB

static __device__ __align__(256) double g_dz_scratch[DZ_STATIC_DOUBLES];

// out[p][0..7] = sum over the G partials of position p (fixed order)
__global__ void k_dz_static_reduce(const double* __restrict__ part, int G, double* __restrict__ out) {
    const int p = blockIdx.x, q = threadIdx.x;
    if (q >= 8) return;
    double s = 0.0;
    for (int g = 0; g < G; ++g) s += part[((int64_t)p * G + g) * 8 + q];
    out[(int64_t)p * 8 + q] = s;
}

double* dz_static_scratch() {
    // the device address of g_dz_scratch, looked up once per device with that device current
    static std::mutex mu;
    static double* addr[64] = {nullptr};
    int dev = 0;
    ECT_CUDA(cudaGetDevice(&dev));
    ECT_REQUIRE(dev >= 0 && dev < 64, ECT_ERR_ARG, "device index out of range");
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        ECT_CUDA(cudaGetSymbolAddress(&p, g_dz_scratch));
        addr[dev] = static_cast<double*>(p);
    }
    return addr[dev];
}

}  // namespace

extern "C" int ect_delta_z_static(ect_ctx* c, const void* d_u0, const void* d_ud, const void* d_b,
                                  const double* h_current, int n_pos, double* h_dz, double* h_dz_emf) {
    if (!c) return ECT_ERR_ARG;
    return guarded_call(c, [&] {
        ECT_REQUIRE(c->mesh_set && c->physics_set, ECT_ERR_STATE, "mesh and physics must be set");
        ECT_REQUIRE(d_u0 && d_ud && h_current && h_dz, ECT_ERR_ARG, "null argument");
        ECT_REQUIRE(n_pos >= 1, ECT_ERR_ARG, "n_pos must be >= 1");
        ECT_REQUIRE(n_pos <= DZ_STATIC_MAX_POS, ECT_ERR_ARG,
                    "ect_delta_z_static handles at most 64 positions per call (its static scratch size)");
        ECT_REQUIRE(!h_dz_emf || d_b, ECT_ERR_ARG, "h_dz_emf needs d_b");
        ECT_REQUIRE(h_current[0] != 0.0 && h_current[1] != 0.0, ECT_ERR_ARG, "coil currents must be non-zero");
        ECT_REQUIRE(!c->mat[0].ibc && !c->mat[1].ibc, ECT_ERR_STATE,
                    "with the impedance boundary condition use ect_delta_z (EMF form)");
        double* base = dz_static_scratch();
        double* part = base;                                              // [n_pos][G][8]
        double* parte = base + (int64_t)DZ_STATIC_MAX_POS * DZ_STATIC_G * 8;  // [n_pos][Ge][8]
        double* res = base + DZ_STATIC_PART;                              // [n_pos][8] then [n_pos][8]
        double* rese = res + (int64_t)DZ_STATIC_MAX_POS * 8;
        cudaStream_t st = c->stream;
        const int64_t nvec = 4 * c->n_nodes;
        k_delta_z<<<dim3(DZ_STATIC_G, n_pos), DZ_TPB, 0, st>>>(
            c->omega_d.as<int32_t>(), c->n_omega_d, c->tets.as<int32_t>(), c->geo.as<double>(),
            c->mat[0].sigma.as<double>(), c->mat[0].nu.as<double>(), c->mat[1].sigma.as<double>(),
            c->mat[1].nu.as<double>(), c->omega, c->delta, (const double2*)d_u0, (const double2*)d_ud, nvec, part);
        ECT_CHECK_LAUNCH();
        k_dz_static_reduce<<<n_pos, 32, 0, st>>>(part, DZ_STATIC_G, res);
        ECT_CHECK_LAUNCH();
        if (h_dz_emf) {
            k_emf<<<dim3(DZ_STATIC_GE, n_pos), 256, 0, st>>>((const double2*)d_b, (const double2*)d_u0,
                                                            (const double2*)d_ud, nvec, parte);
            ECT_CHECK_LAUNCH();
            k_dz_static_reduce<<<n_pos, 32, 0, st>>>(parte, DZ_STATIC_GE, rese);
            ECT_CHECK_LAUNCH();
        }
        // the sums land directly in the caller's host arrays, then get scaled in place
        ECT_CUDA(cudaMemcpyAsync(h_dz, res, sizeof(double) * 8 * n_pos, cudaMemcpyDeviceToHost, st));
        if (h_dz_emf)
            ECT_CUDA(cudaMemcpyAsync(h_dz_emf, rese, sizeof(double) * 8 * n_pos, cudaMemcpyDeviceToHost, st));
        ECT_CUDA(cudaStreamSynchronize(st));
        const double om = c->omega;
        for (int p = 0; p < n_pos; ++p)
            for (int kl = 0; kl < 4; ++kl) {
                const int kk = kl >> 1, l = kl & 1;
                const double f = om / (h_current[kk] * h_current[l]);
                double* z = h_dz + (int64_t)p * 8 + 2 * kl;
                const double sr = z[0], si = z[1];
                z[0] = -f * si;  // (i omega / (I_k I_l)) (sr + i si)
                z[1] = f * sr;
                if (h_dz_emf) {
                    double* e = h_dz_emf + (int64_t)p * 8 + 2 * kl;
                    const double er = e[0], ei = e[1];
                    e[0] = f * ei;  // -(i omega / (I_k I_l)) (er + i ei)
                    e[1] = -f * er;
                }
            }
    });
}
