// Step 2 of the paper's method (Sec. 3): partition the mesh into subdomains.
//
// The paper partitions with Scotch into one subdomain per MPI process.  Here
// the subdomains are small (at most 16 nodes): they are the dense blocks of
// the preconditioner and the first aggregates of the multigrid hierarchy,
// and every subdomain must be a contiguous range of node indices.  Meshes
// that come without such a partition (unstructured meshes from a mesh
// generator) are partitioned by recursive coordinate bisection: a set of
// more than s nodes is cut at the plane normal to the longest side of its
// bounding box into two sets whose sizes are proportional to the numbers of
// blocks they will hold (so no block exceeds s nodes), and the blocks are
// numbered in the order of the recursion, which keeps neighbouring blocks
// close in the numbering (the staged SpMM's tiles of consecutive rows then
// cover compact pieces of the mesh).  Ties in the coordinate are broken by
// node index, and nodes inside a block keep their relative order, so the
// result is deterministic.  Host code only.
#include <algorithm>
#include <numeric>

#include "common.cuh"

namespace {

struct Rcb {
    const double* xyz;
    int s;
    std::vector<int32_t> idx;
    std::vector<int32_t> block_start;

    void run(int64_t lo, int64_t hi) {
        const int64_t n = hi - lo;
        if (n <= s) {
            std::sort(idx.begin() + lo, idx.begin() + hi);
            block_start.push_back((int32_t)lo);
            return;
        }
        const int64_t nb = (n + s - 1) / s, nbl = nb / 2;
        const int64_t nl = n * nbl / nb;  // left: nbl blocks, right: nb - nbl blocks, each <= s nodes
        double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
        for (int64_t e = lo; e < hi; ++e)
            for (int a = 0; a < 3; ++a) {
                const double v = xyz[3 * (int64_t)idx[e] + a];
                mn[a] = std::min(mn[a], v);
                mx[a] = std::max(mx[a], v);
            }
        int ax = 0;
        for (int a = 1; a < 3; ++a)
            if (mx[a] - mn[a] > mx[ax] - mn[ax]) ax = a;
        const double* X = xyz;
        std::nth_element(idx.begin() + lo, idx.begin() + lo + nl, idx.begin() + hi, [X, ax](int32_t p, int32_t q) {
            const double a = X[3 * (int64_t)p + ax], b = X[3 * (int64_t)q + ax];
            return a < b || (a == b && p < q);
        });
        run(lo, lo + nl);
        run(lo + nl, hi);
    }
};

}  // namespace

void partition_rcb(const double* xyz, int64_t n_nodes, int s, int32_t* new_id, int32_t* block_of_new) {
    ECT_REQUIRE(xyz && new_id && block_of_new, ECT_ERR_ARG, "null partition argument");
    ECT_REQUIRE(n_nodes > 0 && n_nodes < (1ll << 30), ECT_ERR_ARG, "n_nodes must be in [1, 2^30)");
    ECT_REQUIRE(s >= 1 && s <= 16, ECT_ERR_ARG, "max_block_nodes must be in [1, 16]");
    for (int64_t e = 0; e < 3 * n_nodes; ++e) ECT_REQUIRE(std::isfinite(xyz[e]), ECT_ERR_MESH, "non-finite coordinate");
    Rcb r{xyz, s, std::vector<int32_t>(n_nodes), {}};
    std::iota(r.idx.begin(), r.idx.end(), 0);
    r.run(0, n_nodes);
    r.block_start.push_back((int32_t)n_nodes);
    for (size_t b = 0; b + 1 < r.block_start.size(); ++b) {
        ECT_REQUIRE(r.block_start[b + 1] - r.block_start[b] <= s, ECT_ERR_ARG, "partition block too large (internal)");
        for (int32_t j = r.block_start[b]; j < r.block_start[b + 1]; ++j) {
            new_id[r.idx[j]] = j;
            block_of_new[j] = (int32_t)b;
        }
    }
}
