// Impedance boundary condition on the support-plate surface (Sec. 2, Eq. IBC
// with the surface integral of Eq. ibcROTA).
//
// The plate (a good conductor whose skin depth delta = sqrt(2/(omega mu_p
// sigma_p)) is small) is removed from the computational domain: its tets
// carry no volume form, every dof of a node that touches only plate tets is
// fixed to zero, and on the plate's surface Gamma_p (faces shared by a plate
// tet and a remaining tet) the A-A block receives
//     -(i omega / Z) int_Gamma A_tau . Phi_tau ds,   Z = (1 - i)/(delta sigma_p),
// with n the unit normal pointing into the plate and A_tau = A - (A.n) n.
// For a surface triangle F and its nodes a, b this is
//     -(i omega / Z) |F| (1 + d_ab)/12 (d_ij - n_i n_j),
// and -(i omega / Z) = (omega delta sigma_p / 2)(1 - i).  V is not carried on
// Gamma_p (it lives on the conducting nodes of the remaining domain), so
// Eq. ibcNORM adds nothing.  Set-up here (host): the surface faces, their
// geometry, and per matrix block the list of (face, a, b) contributions,
// so that the assembly kernel adds them race-free in a fixed order.
#include <algorithm>
#include <array>
#include <cmath>

#include "common.cuh"

namespace {

// local node triples of the four faces of a tet; face f is opposite node f
constexpr int FACE[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

struct FaceRec {
    std::array<int32_t, 3> key;  // sorted node ids
    int32_t tet;
    int8_t f;
    bool operator<(const FaceRec& o) const { return key < o.key || (key == o.key && tet < o.tet); }
};

}  // namespace

void set_ibc(ect_ctx* c, int which, const uint8_t* plate, double sigma_p, double nu_p) {
    ECT_REQUIRE(c->mesh_set, ECT_ERR_STATE, "ect_set_mesh must come first");
    ECT_REQUIRE(which == ECT_VACUUM || which == ECT_DEFECT, ECT_ERR_ARG, "which must be ECT_VACUUM or ECT_DEFECT");
    Matrix& M = c->mat[which];
    const int64_t N = c->n_nodes, T = c->n_tets;
    cudaStream_t st = c->stream;
    clear_sweep(c);
    mg_free(M);
    M.assembled = M.pc_f64 = M.pc_f32 = false;
    if (!plate) {  // clear
        M.ibc = false;
        M.h_void.clear();
        M.n_faces = 0;
        for (DevBuf* b : {&M.tvoid, &M.s_ptr, &M.s_ent, &M.s_geo}) b->release();
        std::vector<double> s = M.h_sigma, n = M.h_nu;
        upload_config(c, which, s, n);
        return;
    }
    ECT_REQUIRE(std::isfinite(sigma_p) && sigma_p > 0.0 && std::isfinite(nu_p) && nu_p > 0.0, ECT_ERR_ARG,
                "plate sigma and nu must be finite and > 0");
    const int32_t* tet = c->h_tets.data();
    const double* X = nullptr;
    std::vector<double> hxyz(3 * N);
    ECT_CUDA(cudaMemcpyAsync(hxyz.data(), c->xyz.p, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, st));
    ECT_CUDA(cudaStreamSynchronize(st));
    X = hxyz.data();
    // faces of plate tets, and faces of other tets whose three nodes all touch the plate
    std::vector<uint8_t> pnode(N, 0);
    int64_t n_plate = 0;
    for (int64_t t = 0; t < T; ++t)
        if (plate[t]) {
            ++n_plate;
            for (int a = 0; a < 4; ++a) pnode[tet[4 * t + a]] = 1;
        }
    ECT_REQUIRE(n_plate > 0 && n_plate < T, ECT_ERR_ARG, "the plate must be a proper, non-empty subset of the tets");
    std::vector<FaceRec> pf, of;
    for (int64_t t = 0; t < T; ++t)
        for (int8_t f = 0; f < 4; ++f) {
            FaceRec r{{tet[4 * t + FACE[f][0]], tet[4 * t + FACE[f][1]], tet[4 * t + FACE[f][2]]}, (int32_t)t, f};
            if (!plate[t] && !(pnode[r.key[0]] && pnode[r.key[1]] && pnode[r.key[2]])) continue;
            std::sort(r.key.begin(), r.key.end());
            (plate[t] ? pf : of).push_back(r);
        }
    std::sort(pf.begin(), pf.end());
    std::sort(of.begin(), of.end());
    // merge: a plate face that is also a face of a remaining tet lies on Gamma_p
    std::vector<std::array<int32_t, 3>> tri;
    std::vector<double> geo;
    size_t j = 0;
    for (size_t i = 0; i < pf.size(); ++i) {
        while (j < of.size() && of[j].key < pf[i].key) ++j;
        if (j == of.size() || of[j].key != pf[i].key) continue;
        const int32_t t = pf[i].tet;
        const int f = pf[i].f;
        const int32_t v0 = tet[4 * t + FACE[f][0]], v1 = tet[4 * t + FACE[f][1]], v2 = tet[4 * t + FACE[f][2]];
        const int32_t opp = tet[4 * t + f];
        double e1[3], e2[3], nrm[3], w[3];
        for (int a = 0; a < 3; ++a) {
            e1[a] = X[3 * (int64_t)v1 + a] - X[3 * (int64_t)v0 + a];
            e2[a] = X[3 * (int64_t)v2 + a] - X[3 * (int64_t)v0 + a];
            w[a] = X[3 * (int64_t)opp + a] - X[3 * (int64_t)v0 + a];
        }
        nrm[0] = e1[1] * e2[2] - e1[2] * e2[1];
        nrm[1] = e1[2] * e2[0] - e1[0] * e2[2];
        nrm[2] = e1[0] * e2[1] - e1[1] * e2[0];
        const double len = std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
        ECT_REQUIRE(len > 0.0, ECT_ERR_MESH, "degenerate plate face");
        double sgn = (nrm[0] * w[0] + nrm[1] * w[1] + nrm[2] * w[2]) < 0.0 ? -1.0 : 1.0;  // into the plate tet
        tri.push_back({v0, v1, v2});
        geo.push_back(0.5 * len);
        for (int a = 0; a < 3; ++a) geo.push_back(sgn * nrm[a] / len);
    }
    const int64_t F = (int64_t)tri.size();
    ECT_REQUIRE(F > 0, ECT_ERR_ARG, "the plate has no face shared with the rest of the mesh");
    ECT_REQUIRE(F < (1ll << 27), ECT_ERR_ARG, "too many plate faces");
    // per block: its (face, a, b) contributions, in face order
    const std::vector<int32_t>& rp = c->h_row_ptr;
    const std::vector<int32_t>& cl = c->h_col;
    std::vector<std::pair<int32_t, uint32_t>> ent;
    ent.reserve(9 * F);
    for (int64_t f = 0; f < F; ++f)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                const int32_t r = tri[f][a], col = tri[f][b];
                const int32_t* lo = cl.data() + rp[r];
                const int32_t* hi = cl.data() + rp[r + 1];
                const int32_t* it = std::lower_bound(lo, hi, col);
                ECT_REQUIRE(it != hi && *it == col, ECT_ERR_MESH, "plate face outside the block pattern (internal)");
                ent.emplace_back((int32_t)(it - cl.data()), (uint32_t)(f << 4 | a << 2 | b));
            }
    std::stable_sort(ent.begin(), ent.end(),
                     [](const std::pair<int32_t, uint32_t>& x, const std::pair<int32_t, uint32_t>& y) {
                         return x.first < y.first;
                     });
    std::vector<int32_t> sptr(c->nnzb + 1, 0);
    std::vector<uint32_t> sent(ent.size());
    for (size_t e = 0; e < ent.size(); ++e) {
        ++sptr[ent[e].first + 1];
        sent[e] = ent[e].second;
    }
    for (int64_t s = 0; s < c->nnzb; ++s) sptr[s + 1] += sptr[s];
    M.ibc = true;
    M.ibc_sigma = sigma_p;
    M.ibc_nu = nu_p;
    M.h_void.assign(plate, plate + T);
    M.n_faces = F;
    auto up = [&](DevBuf& d, const void* h, size_t bytes) {
        d.alloc(bytes);
        ECT_CUDA(cudaMemcpyAsync(d.p, h, bytes, cudaMemcpyHostToDevice, st));
    };
    up(M.tvoid, M.h_void.data(), T);
    up(M.s_ptr, sptr.data(), sizeof(int32_t) * sptr.size());
    up(M.s_ent, sent.data(), sizeof(uint32_t) * sent.size());
    up(M.s_geo, geo.data(), sizeof(double) * geo.size());
    std::vector<double> s = M.h_sigma, n = M.h_nu;
    upload_config(c, which, s, n);  // constraint mask with the plate removed (synchronises)
}
