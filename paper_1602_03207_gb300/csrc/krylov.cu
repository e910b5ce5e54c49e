// Kernel (d) and the solver drivers: restarted flexible GMRES for k
// right-hand sides in lockstep.
//
// The paper factorises once and solves one right-hand side per probe
// position (Sec. 3, Steps 5-6).  Here the solve is Krylov: right-
// preconditioned flexible GMRES (Saad) on the scaled system S y = T b,
// x = T y, S = T M T, with the subdomain-block preconditioner.  Every
// right-hand side has its own basis, Hessenberg matrix and Givens rotations;
// all of them advance together in the same kernels, and one that has met the
// tolerance is skipped by every later kernel of the cycle.
//
// Arnoldi step (classical Gram-Schmidt applied twice, Hermitian product):
//   h1 = V^H w, w -= V h1, h2 = V^H w, w -= V h2, H(:,j) = h1 + h2,
//   H(j+1,j) = ||w||, v_{j+1} = w / ||w||,
// built from a multi-vector dot (per-CTA partial sums with warp shuffles,
// then a fixed-order reduction, so results are bitwise reproducible), a
// kernel that applies the first update and forms the second pass's dots and
// ||w||^2 in the same pass over the basis (up to 12 vectors in FP32, 8 in
// FP64; two separate passes beyond), a multi-vector axpy that also
// accumulates ||w||^2, and a
// per-right-hand-side finalize kernel that applies the previous Givens
// rotations to the new column, forms the next rotation, updates the
// residual estimate |g_{j+1}| and retires converged right-hand sides.
//
// Mixed mode: the outer loop is the FP64 flexible GMRES above; its
// preconditioner is a fixed number of FP32 GMRES iterations (right-
// preconditioned by the FP32 subdomain blocks, FP32 SpMV and vectors, FP64
// Hessenberg/Givens) started from zero on S z = v_j; the preconditioned
// inner vectors P^-1 v_i are kept, so the inner solution is their
// combination and needs no further preconditioner application.  The FP64 outer loop
// keeps the residual, its orthogonalisation and least-squares problem in
// FP64, so the final accuracy is that of FP64.
//
// A restart cycle is a fixed sequence of launches; with use_graph it is
// captured once into a CUDA graph and replayed.  The host reads back the k
// true residual norms only at restart boundaries.
#include <chrono>
#include <cmath>
#include <map>
#include <tuple>
#include <type_traits>

#include "common.cuh"

namespace {

constexpr int TPB = 256;
constexpr int GV = 8;  // basis vectors per pass of the multi-dot

template <typename T> __device__ __forceinline__ C<T> ldc(const C<T>* p) { return *p; }

// block-wide sum of NV doubles held by every thread; result valid in thread 0
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh /* [8][NV] */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) sh[warp * NV + q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += sh[w * NV + q];
            v[q] = s;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void chunk_range(int64_t n, int G, int g, int64_t& lo, int64_t& hi) {
    int64_t per = (n + G - 1) / G;
    per = (per + TPB - 1) / TPB * TPB;
    lo = (int64_t)g * per;
    hi = lo + per;
    if (hi > n) hi = n;
}

// One group of NQ basis vectors of the multi-dot.  The vector indices are
// clamped to the last one, so every load is unconditional and the loads of a
// step issue together (predicated loads would be serialised by branches); the
// partial sums of the clamped duplicates are computed and never stored.
template <typename T, int NQ>
__device__ __forceinline__ void mdot_group(const C<T>* __restrict__ vr, int64_t vstride, int i0, int nvec,
                                           const C<T>* __restrict__ w, int64_t lo, int64_t hi, C<T> (&acc)[GV],
                                           T& wn) {
    const C<T>* vq[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) vq[q] = vr + (int64_t)(i0 + q < nvec ? i0 + q : nvec - 1) * vstride;
#pragma unroll 2  // independent elements: more loads in flight
    for (int64_t e = lo + threadIdx.x; e < hi; e += TPB) {
        const C<T> we = w[e];
        wn += we.x * we.x + we.y * we.y;
#pragma unroll
        for (int q = 0; q < NQ; ++q) cfma_conj(acc[q], vq[q][e], we);
    }
}

// part[(r*nvec + i)*G + g] = sum over this CTA's range of conj(V_i[r][e]) * W[r][e]
// and, when wpart is given, wpart[r*G + g] = sum of |W[r][e]|^2 over the range
template <typename T>
__global__ void __launch_bounds__(TPB) k_mdot(const C<T>* __restrict__ V, int64_t vstride, int nvec,
                                              const C<T>* __restrict__ W, int64_t ld, int64_t n,
                                              const int* __restrict__ live, double2* __restrict__ part, int G,
                                              double* __restrict__ wpart) {
    __shared__ double sh[8 * (2 * GV + 1)];
    const int r = blockIdx.y, g = blockIdx.x;
    if (live && !live[r]) return;
    int64_t lo, hi;
    chunk_range(n, G, g, lo, hi);
    const C<T>* w = W + (int64_t)r * ld;
    const C<T>* vr = V + (int64_t)r * ld;
    for (int i0 = 0; i0 < nvec; i0 += GV) {
        C<T> acc[GV];
        T wn = T(0);
#pragma unroll
        for (int q = 0; q < GV; ++q) acc[q] = czero<T>();
        if (nvec - i0 > GV / 2) mdot_group<T, GV>(vr, vstride, i0, nvec, w, lo, hi, acc, wn);
        else mdot_group<T, GV / 2>(vr, vstride, i0, nvec, w, lo, hi, acc, wn);
        double s[2 * GV + 1];
#pragma unroll
        for (int q = 0; q < GV; ++q) {
            s[2 * q] = (double)acc[q].x;
            s[2 * q + 1] = (double)acc[q].y;
        }
        s[2 * GV] = (double)wn;
        block_sum<2 * GV + 1>(s, sh);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int q = 0; q < GV; ++q)
                if (i0 + q < nvec) part[((int64_t)r * nvec + i0 + q) * G + g] = make_double2(s[2 * q], s[2 * q + 1]);
            if (wpart && i0 == 0) wpart[(int64_t)r * G + g] = s[2 * GV];
        }
    }
}

// First Gram-Schmidt update fused with the dot products of the second pass.
// W[r] -= sum_i hp[r][i] V_i[r] (the operations of k_maxpy in the same order),
// then, on the updated W, part[(r*nvec + i)*G + g] = sum conj(V_i[r][e]) W[r][e]
// and npart[r*G + g] = sum |W[r][e]|^2 over this CTA's range (the operations of
// k_mdot and k_norm_part in the same order).  The V_i[r][e] are loaded once and
// reused from registers: the pair costs one pass over the basis instead of two.
template <typename T, int NV>
__global__ void __launch_bounds__(TPB, 2) k_maxpy_mdot(const C<T>* __restrict__ V, int64_t vstride, int nvec,
                                                       C<T>* __restrict__ W, int64_t ld, int64_t n,
                                                       const double2* __restrict__ hp, int ldp,
                                                       const int* __restrict__ live, double2* __restrict__ part,
                                                       double* __restrict__ npart, int G) {
    __shared__ C<T> hs[NV];
    __shared__ double sh[8 * (2 * GV + 1)];
    const int r = blockIdx.y, g = blockIdx.x;
    if (live && !live[r]) return;
    for (int i = threadIdx.x; i < NV; i += TPB) {
        const double2 h = i < nvec ? hp[(int64_t)r * ldp + i] : make_double2(0.0, 0.0);
        hs[i] = from_d<T>(make_double2(-h.x, -h.y));  // zero beyond nvec: the padded terms add nothing
    }
    __syncthreads();
    int64_t lo, hi;
    chunk_range(n, G, g, lo, hi);
    C<T>* w = W + (int64_t)r * ld;
    const C<T>* vr = V + (int64_t)r * ld;
    C<T> acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = czero<T>();
    T nacc = T(0);
    // vector indices clamped to the last one: unconditional loads (see mdot_group)
    const C<T>* vq[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) vq[q] = vr + (int64_t)(q < nvec ? q : nvec - 1) * vstride;
    for (int64_t e = lo + threadIdx.x; e < hi; e += TPB) {
        C<T> v[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] = vq[q][e];
        C<T> we = w[e];
#pragma unroll
        for (int q = 0; q < NV; ++q) cfma(we, hs[q], v[q]);
        w[e] = we;
        nacc += we.x * we.x + we.y * we.y;
#pragma unroll
        for (int q = 0; q < NV; ++q) cfma_conj(acc[q], v[q], we);
    }
    // reduce in groups of GV vectors (bounded register use); the norm rides with the first group
#pragma unroll
    for (int i0 = 0; i0 < NV; i0 += GV) {
        if (i0 > 0 && i0 >= nvec) break;
        double s[2 * GV + 1];
#pragma unroll
        for (int q = 0; q < GV; ++q) {
            const int iq = i0 + q < NV ? i0 + q : 0;  // NV need not be a multiple of GV
            s[2 * q] = i0 + q < NV ? (double)acc[iq].x : 0.0;
            s[2 * q + 1] = i0 + q < NV ? (double)acc[iq].y : 0.0;
        }
        s[2 * GV] = (double)nacc;
        block_sum<2 * GV + 1>(s, sh);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int q = 0; q < GV; ++q)
                if (i0 + q < nvec) part[((int64_t)r * nvec + i0 + q) * G + g] = make_double2(s[2 * q], s[2 * q + 1]);
            if (i0 == 0) npart[(int64_t)r * G + g] = s[2 * GV];
        }
    }
}

// deterministic warp sum of G partials (fixed lane assignment and shuffle tree)
__device__ __forceinline__ double warp_sum_partials(const double* __restrict__ p, int G) {
    double s = 0.0;
    for (int g = threadIdx.x & 31; g < G; g += 32) s += p[g];
    return warp_sum(s);
}

// second Gram-Schmidt pass needed?  live2[r] = live[r] && ||w1||^2 < ||w0||^2 / 2
__global__ void k_reorth_decide(const double* __restrict__ wpart, int Gw, const double* __restrict__ npart, int G,
                                int k, const int* __restrict__ live, int* __restrict__ live2) {
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= k) return;
    if (!live[r]) {
        if ((threadIdx.x & 31) == 0) live2[r] = 0;
        return;
    }
    const double n0 = warp_sum_partials(wpart + (int64_t)r * Gw, Gw);
    const double n1 = warp_sum_partials(npart + (int64_t)r * G, G);
    if ((threadIdx.x & 31) == 0) live2[r] = (n1 < 0.5 * n0) ? 1 : 0;
}

// hp[r*ldp + i] = sum_g part; H[r*ldh + hoff + i] (+)= the same
__global__ void k_dot_reduce(const double2* __restrict__ part, int G, int nvec, int k, const int* __restrict__ live,
                             double2* __restrict__ hp, int ldp, double2* __restrict__ H, int64_t ldh, int64_t hoff,
                             int accumulate) {
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (wid >= k * nvec) return;
    const int r = wid / nvec, i = wid - r * nvec;
    if (live && !live[r]) return;
    double sx = 0.0, sy = 0.0;
    for (int gg = lane; gg < G; gg += 32) {
        double2 v = part[((int64_t)r * nvec + i) * G + gg];
        sx += v.x;
        sy += v.y;
    }
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    if (lane == 0) {
        hp[(int64_t)r * ldp + i] = make_double2(sx, sy);
        if (H) {
            double2* h = H + (int64_t)r * ldh + hoff + i;
            if (accumulate) *h = make_double2(h->x + sx, h->y + sy);
            else *h = make_double2(sx, sy);
        }
    }
}

// W[r] -= sign * sum_i hp[r][i] V_i[r]; optionally norm partials of the result
template <typename T>
__global__ void __launch_bounds__(TPB) k_maxpy(const C<T>* __restrict__ V, int64_t vstride, int nvec,
                                               C<T>* __restrict__ W, int64_t ld, int64_t n,
                                               const double2* __restrict__ hp, int ldp, double sign,
                                               const int* __restrict__ live, double* __restrict__ npart, int G) {
    __shared__ C<T> hs[72];
    __shared__ double sh[8];
    const int r = blockIdx.y, g = blockIdx.x;
    if (live && !live[r]) return;
    for (int i = threadIdx.x; i < nvec; i += TPB) {
        double2 h = hp[(int64_t)r * ldp + i];
        hs[i] = from_d<T>(make_double2(-sign * h.x, -sign * h.y));
    }
    __syncthreads();
    int64_t lo, hi;
    chunk_range(n, G, g, lo, hi);
    C<T>* w = W + (int64_t)r * ld;
    T nacc = T(0);
#pragma unroll 2
    for (int64_t e = lo + threadIdx.x; e < hi; e += TPB) {
        C<T> we = w[e];
        for (int i = 0; i < nvec; ++i) cfma(we, hs[i], V[(int64_t)i * vstride + (int64_t)r * ld + e]);
        w[e] = we;
        nacc += we.x * we.x + we.y * we.y;
    }
    if (npart) {
        double s[1] = {(double)nacc};
        block_sum<1>(s, sh);
        if (threadIdx.x == 0) npart[(int64_t)r * G + g] = s[0];
    }
}

// norm partials of W[r]
template <typename T>
__global__ void __launch_bounds__(TPB) k_norm_part(const C<T>* __restrict__ W, int64_t ld, int64_t n,
                                                   const int* __restrict__ live, double* __restrict__ npart, int G) {
    __shared__ double sh[8];
    const int r = blockIdx.y, g = blockIdx.x;
    if (live && !live[r]) return;
    int64_t lo, hi;
    chunk_range(n, G, g, lo, hi);
    const C<T>* w = W + (int64_t)r * ld;
    T nacc = T(0);
#pragma unroll 4
    for (int64_t e = lo + threadIdx.x; e < hi; e += TPB) {
        C<T> we = w[e];
        nacc += we.x * we.x + we.y * we.y;
    }
    double s[1] = {(double)nacc};
    block_sum<1>(s, sh);
    if (threadIdx.x == 0) npart[(int64_t)r * G + g] = s[0];
}

__global__ void k_norm_finalize(const double* __restrict__ npart, int G, int k, const int* __restrict__ live,
                                double* __restrict__ out) {
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= k) return;
    if (live && !live[r]) return;
    double s = 0.0;
    for (int g = threadIdx.x & 31; g < G; g += 32) s += npart[(int64_t)r * G + g];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) out[r] = sqrt(s);
}

__device__ __forceinline__ void givens(double2 a, double2 b, double& c, double2& s, double2& rr) {
    double ab = hypot(a.x, a.y), bb = hypot(b.x, b.y);
    if (bb == 0.0) {
        c = 1.0;
        s = make_double2(0.0, 0.0);
        rr = a;
        return;
    }
    if (ab == 0.0) {
        c = 0.0;
        s = make_double2(1.0, 0.0);
        rr = b;
        return;
    }
    double rho = hypot(ab, bb);
    double2 ph = make_double2(a.x / ab, a.y / ab);
    c = ab / rho;
    double2 cb = make_double2(b.x / rho, -b.y / rho);  // conj(b)/rho
    s = cmul(ph, cb);
    rr = make_double2(ph.x * rho, ph.y * rho);
}

// Column j of the Hessenberg matrix of every live right-hand side: new
// subdiagonal from the norm partials, previous rotations, new rotation,
// residual estimate and retirement.  flags bit 0: NaN/Inf seen.
__global__ void k_arnoldi_finalize(const double* __restrict__ npart, int G, int k, int j, int m,
                                   double2* __restrict__ H, double* __restrict__ cs, double2* __restrict__ sn,
                                   double2* __restrict__ g, const double* __restrict__ target,
                                   int* __restrict__ live, int* __restrict__ nit, double* __restrict__ inv_h,
                                   int* __restrict__ flags) {
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= k || !live[r]) return;
    double s = 0.0;
    for (int gg = threadIdx.x & 31; gg < G; gg += 32) s += npart[(int64_t)r * G + gg];
    s = warp_sum(s);
    if ((threadIdx.x & 31) != 0) return;
    const double hn = sqrt(s);
    double2* Hc = H + (int64_t)r * (m + 1) * m + (int64_t)j * (m + 1);
    Hc[j + 1] = make_double2(hn, 0.0);
    double* c_ = cs + (int64_t)r * m;
    double2* s_ = sn + (int64_t)r * m;
    double2* g_ = g + (int64_t)r * (m + 1);
    for (int i = 0; i < j; ++i) {
        double2 a = Hc[i], b = Hc[i + 1], si = s_[i];
        double ci = c_[i];
        double2 t = cadd(cscale(a, ci), cmul(si, b));
        double2 sc = make_double2(-si.x, si.y);  // -conj(s)
        Hc[i + 1] = cadd(cmul(sc, a), cscale(b, ci));
        Hc[i] = t;
    }
    double c;
    double2 sv, rr;
    givens(Hc[j], Hc[j + 1], c, sv, rr);
    c_[j] = c;
    s_[j] = sv;
    Hc[j] = rr;
    Hc[j + 1] = make_double2(0.0, 0.0);
    double2 gj = g_[j];
    double2 sc = make_double2(-sv.x, sv.y);
    g_[j + 1] = cmul(sc, gj);
    g_[j] = cscale(gj, c);
    const double res = hypot(g_[j + 1].x, g_[j + 1].y);
    const bool bad = !isfinite(hn) || !isfinite(res) || !isfinite(rr.x) || !isfinite(rr.y);
    if (bad) {
        atomicOr(flags, 1);
        live[r] = 0;
        nit[r] = j;  // drop the broken column
        inv_h[r] = 0.0;
        return;
    }
    nit[r] = j + 1;
    if (res <= target[r] || hn == 0.0 || j + 1 >= m) live[r] = 0;
    inv_h[r] = hn > 0.0 ? 1.0 / hn : 0.0;
}

template <typename T>
__global__ void __launch_bounds__(TPB) k_scale_vec(const C<T>* __restrict__ W, C<T>* __restrict__ Out, int64_t ld,
                                                   int64_t n, const double* __restrict__ f, const int* __restrict__ live,
                                                   int k) {
    const int r = blockIdx.y;
    if (live && !live[r]) return;
    const T s = (T)f[r];
    for (int64_t e = blockIdx.x * (int64_t)TPB + threadIdx.x; e < n; e += (int64_t)gridDim.x * TPB) {
        C<T> v = W[(int64_t)r * ld + e];
        Out[(int64_t)r * ld + e] = cscale(v, s);
    }
}

// start of a cycle: V_0 = R / beta, g = beta e_1
__global__ void k_cycle_g0(const double* __restrict__ rnorm, const int* __restrict__ run, int k, int m,
                           double2* __restrict__ g, double* __restrict__ invb, int* __restrict__ live,
                           int* __restrict__ nit) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= k) return;
    live[r] = run[r];
    nit[r] = 0;
    double b = rnorm[r];
    g[(int64_t)r * (m + 1)] = make_double2(b, 0.0);
    invb[r] = (run[r] && b > 0.0) ? 1.0 / b : 0.0;
}

// inner solve start: live_i = live, g_i = e_1 (the inner start vector has unit norm)
__global__ void k_inner_g0(const int* __restrict__ live, int k, int m, double2* __restrict__ g,
                           int* __restrict__ live_i, int* __restrict__ nit) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= k) return;
    live_i[r] = live[r];
    nit[r] = 0;
    g[(int64_t)r * (m + 1)] = make_double2(1.0, 0.0);
}

// back substitution H(0:n,0:n) y = g(0:n) with n = nit[r]
__global__ void k_trisolve(const double2* __restrict__ H, const double2* __restrict__ g, const int* __restrict__ nit,
                           const int* __restrict__ run, int k, int m, double2* __restrict__ y) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= k) return;
    double2* yr = y + (int64_t)r * (m + 1);
    const int nn = run[r] ? nit[r] : 0;
    for (int i = nn; i <= m; ++i) yr[i] = make_double2(0.0, 0.0);
    const double2* Hr = H + (int64_t)r * (m + 1) * m;
    const double2* gr = g + (int64_t)r * (m + 1);
    for (int i = nn - 1; i >= 0; --i) {
        double2 s = gr[i];
        for (int jj = i + 1; jj < nn; ++jj) s = csub(s, cmul(Hr[(int64_t)jj * (m + 1) + i], yr[jj]));
        double2 d = Hr[(int64_t)i * (m + 1) + i];
        double dd = d.x * d.x + d.y * d.y;
        yr[i] = dd > 0.0 ? make_double2((s.x * d.x + s.y * d.y) / dd, (s.y * d.x - s.x * d.y) / dd)
                         : make_double2(0.0, 0.0);
    }
}

// R[r] = B[r] - R[r] with norm partials
__global__ void __launch_bounds__(TPB) k_residual(const double2* __restrict__ B, double2* __restrict__ R, int64_t ld,
                                                  int64_t n, const int* __restrict__ run, double* __restrict__ npart,
                                                  int G) {
    __shared__ double sh[8];
    const int r = blockIdx.y, g = blockIdx.x;
    if (!run[r]) return;
    int64_t lo, hi;
    chunk_range(n, G, g, lo, hi);
    double nacc = 0.0;
    for (int64_t e = lo + threadIdx.x; e < hi; e += TPB) {
        double2 v = csub(B[(int64_t)r * ld + e], R[(int64_t)r * ld + e]);
        R[(int64_t)r * ld + e] = v;
        nacc += v.x * v.x + v.y * v.y;
    }
    double s[1] = {nacc};
    block_sum<1>(s, sh);
    if (threadIdx.x == 0) npart[(int64_t)r * G + g] = s[0];
}

__global__ void k_d2f(const double2* __restrict__ a, float2* __restrict__ b, int64_t ld, int64_t n,
                      const int* __restrict__ live) {
    const int r = blockIdx.y;
    if (live && !live[r]) return;
    for (int64_t e = blockIdx.x * (int64_t)TPB + threadIdx.x; e < n; e += (int64_t)gridDim.x * TPB) {
        double2 v = a[(int64_t)r * ld + e];
        b[(int64_t)r * ld + e] = make_float2((float)v.x, (float)v.y);
    }
}

__global__ void k_f2d(const float2* __restrict__ a, double2* __restrict__ b, int64_t ld, int64_t n,
                      const int* __restrict__ live) {
    const int r = blockIdx.y;
    if (live && !live[r]) return;
    for (int64_t e = blockIdx.x * (int64_t)TPB + threadIdx.x; e < n; e += (int64_t)gridDim.x * TPB) {
        float2 v = a[(int64_t)r * ld + e];
        b[(int64_t)r * ld + e] = make_double2(v.x, v.y);
    }
}

// out[r][e] = t[e] * in[r][e]  (in/out unscaled <-> scaled)
__global__ void k_diag_scale(const double2* __restrict__ in, double2* __restrict__ out, const double* __restrict__ t,
                             int64_t ld, int64_t n) {
    const int r = blockIdx.y;
    for (int64_t e = blockIdx.x * (int64_t)TPB + threadIdx.x; e < n; e += (int64_t)gridDim.x * TPB)
        out[(int64_t)r * ld + e] = cscale(in[(int64_t)r * ld + e], t[e]);
}

// out = in / t elementwise (t > 0: the scaling of the system)
__global__ void k_diag_unscale(const double2* __restrict__ in, double2* __restrict__ out, const double* __restrict__ t,
                               int64_t ld, int64_t n) {
    const int r = blockIdx.y;
    for (int64_t e = blockIdx.x * (int64_t)TPB + threadIdx.x; e < n; e += (int64_t)gridDim.x * TPB) {
        const double2 v = in[(int64_t)r * ld + e];
        const double it = 1.0 / t[e];
        out[(int64_t)r * ld + e] = make_double2(v.x * it, v.y * it);
    }
}

template <typename T>
__global__ void k_zero(C<T>* __restrict__ a, int64_t ld, int64_t n, const int* __restrict__ live) {
    const int r = blockIdx.y;
    if (live && !live[r]) return;
    for (int64_t e = blockIdx.x * (int64_t)TPB + threadIdx.x; e < n; e += (int64_t)gridDim.x * TPB)
        a[(int64_t)r * ld + e] = czero<T>();
}

}  // namespace

// ----------------------------------------------------------------------------
// workspace
// ----------------------------------------------------------------------------
struct Workspace {
    int k = 0, m = 0, mi = 0, mode = -1;
    int64_t n = 0;
    int G = 1;
    DevBuf V, Z, Y, Bh, R;
    DevBuf V32, U32, Z32;
    DevBuf H, cs, sn, g, y, hp;
    DevBuf Hi, csi, sni, gi, yi;
    DevBuf part, npart, wpart;
    DevBuf bnorm, rnorm, target, target_i, inv_h, invb, run, live, live_i, nit, nit_i, flags, live2;
    bool selective = true;
    bool inner_one_pass = false;  // mixed mode: one classical Gram-Schmidt pass in the FP32 loop
    bool outer_one_pass = false;  // one classical Gram-Schmidt pass in the FP64 loop
    std::map<std::tuple<int, int, int, int, int>, std::pair<cudaGraphExec_t, size_t>> graphs;  // exec, kernel nodes
    ~Workspace() {
        for (auto& kv : graphs) cudaGraphExecDestroy(kv.second.first);
    }
};

void workspace_free(ect_ctx* c) {
    delete c->ws;
    c->ws = nullptr;
}

namespace {

int pick_G(int64_t n, int k) {
    int64_t G = (n + 4095) / 4096;
    int64_t cap = std::max<int64_t>(1, 1216 / std::max(1, k));
    if (G > cap) G = cap;
    if (G < 1) G = 1;
    return (int)G;
}

Workspace* get_ws(ect_ctx* c, int k, int m, int mi, int mode) {
    const int64_t n = 4 * c->n_nodes;
    Workspace* w = c->ws;
    if (w && w->k == k && w->m == m && w->mi == mi && w->mode == mode && w->n == n) return w;
    workspace_free(c);
    w = new Workspace();
    c->ws = w;
    w->k = k;
    w->m = m;
    w->mi = mi;
    w->mode = mode;
    w->n = n;
    w->G = pick_G(n, k);
    const size_t vec = sizeof(double2) * (size_t)n * k;
    w->V.alloc(vec * (m + 1));
    w->Z.alloc(vec * m);
    w->Y.alloc(vec);
    w->Bh.alloc(vec);
    w->R.alloc(vec);
    const int mm = std::max(m, mi);
    w->H.alloc(sizeof(double2) * (size_t)k * (m + 1) * m);
    w->cs.alloc(sizeof(double) * (size_t)k * m);
    w->sn.alloc(sizeof(double2) * (size_t)k * m);
    w->g.alloc(sizeof(double2) * (size_t)k * (m + 1));
    w->y.alloc(sizeof(double2) * (size_t)k * (m + 1));
    w->hp.alloc(sizeof(double2) * (size_t)k * (mm + 1));
    if (mode == ECT_MODE_MIXED) {
        const size_t vec32 = sizeof(float2) * (size_t)n * k;
        w->V32.alloc(vec32 * (mi + 1));
        w->U32.alloc(vec32);
        w->Z32.alloc(vec32 * mi);
        // the combination below multiplies unused entries by zero: keep them finite
        ECT_CUDA(cudaMemset(w->Z32.p, 0, w->Z32.bytes));
        w->Hi.alloc(sizeof(double2) * (size_t)k * (mi + 1) * mi);
        w->csi.alloc(sizeof(double) * (size_t)k * mi);
        w->sni.alloc(sizeof(double2) * (size_t)k * mi);
        w->gi.alloc(sizeof(double2) * (size_t)k * (mi + 1));
        w->yi.alloc(sizeof(double2) * (size_t)k * (mi + 1));
    }
    w->part.alloc(sizeof(double2) * (size_t)k * (mm + 1) * w->G);
    w->npart.alloc(sizeof(double) * (size_t)k * w->G);
    w->wpart.alloc(sizeof(double) * (size_t)k * w->G);
    w->live2.alloc(sizeof(int) * k);
    for (DevBuf* b : {&w->bnorm, &w->rnorm, &w->target, &w->target_i, &w->inv_h, &w->invb})
        b->alloc(sizeof(double) * k);
    for (DevBuf* b : {&w->run, &w->live, &w->live_i, &w->nit, &w->nit_i}) b->alloc(sizeof(int) * k);
    w->flags.alloc(sizeof(int));
    return w;
}

inline dim3 vgrid(const Workspace* w) { return dim3((unsigned)w->G, (unsigned)w->k); }

inline unsigned ew_blocks(int64_t n, int k) {
    int64_t b = (n + TPB - 1) / TPB;
    int64_t cap = std::max<int64_t>(1, 4096 / std::max(1, k));
    return (unsigned)std::max<int64_t>(1, std::min(b, cap));
}

// one CGS2 Arnoldi step on basis vectors V_0..V_j (storage T), new vector W
template <typename T>
void cgs2_step(ect_ctx* c, Workspace* w, const C<T>* V, int64_t vstride, int j, C<T>* W, int64_t ld,
               double2* H, int m, const int* live, bool one_pass = false) {
    cudaStream_t st = c->stream;
    const int nvec = j + 1, k = w->k, G = w->G;
    const int64_t n = w->n;
    double2* part = w->part.as<double2>();
    double2* hp = w->hp.as<double2>();
    const int ldp = std::max(w->m, w->mi) + 1;
    const int64_t ldh = (int64_t)(m + 1) * m, hoff = (int64_t)j * (m + 1);
    const unsigned rb = grid_for((int64_t)k * nvec * 32, 256);
    const bool sel = w->selective && live != nullptr;
    double* npart = w->npart.as<double>();
    const dim3 vg = vgrid(w);
    // pass 1: h1 = V^H w
    k_mdot<T><<<vg, TPB, 0, st>>>(V, vstride, nvec, W, ld, n, live, part, G, sel ? w->wpart.as<double>() : nullptr);
    k_dot_reduce<<<rb, 256, 0, st>>>(part, G, nvec, k, live, hp, ldp, H, ldh, hoff, 0);
    if (one_pass) {
        // classical Gram-Schmidt: w -= V h1 and ||w||^2, no second pass
        k_maxpy<T><<<vg, TPB, 0, st>>>(V, vstride, nvec, W, ld, n, hp, ldp, 1.0, live, npart, G);
        ECT_CHECK_LAUNCH();
        return;
    }
    // w1 = w - V h1, fused with h2 = V^H w1 and ||w1||^2 when the basis fits the register tile
    // (12 vectors in FP32, 8 in FP64: beyond that the registers spill or cut occupancy below the
    // two-pass cost)
    bool fused = true;
    constexpr bool f32 = std::is_same<T, float>::value;
    if (nvec <= 4)
        k_maxpy_mdot<T, 4><<<vg, TPB, 0, st>>>(V, vstride, nvec, W, ld, n, hp, ldp, live, part, npart, G);
    else if (nvec <= 8)
        k_maxpy_mdot<T, 8><<<vg, TPB, 0, st>>>(V, vstride, nvec, W, ld, n, hp, ldp, live, part, npart, G);
    else if (f32 && nvec <= 12)
        k_maxpy_mdot<T, f32 ? 12 : 8><<<vg, TPB, 0, st>>>(V, vstride, nvec, W, ld, n, hp, ldp, live, part, npart, G);
    else {
        fused = false;
        k_maxpy<T><<<vg, TPB, 0, st>>>(V, vstride, nvec, W, ld, n, hp, ldp, 1.0, live, sel ? npart : nullptr, G);
    }
    // pass 2 (for the right-hand sides that need it when selective): w2 = w1 - V h2
    const int* live2 = live;
    if (sel) {
        k_reorth_decide<<<grid_for((int64_t)k * 32, 128), 128, 0, st>>>(w->wpart.as<double>(), G, npart, G, k, live,
                                                                        w->live2.as<int>());
        live2 = w->live2.as<int>();
    }
    if (!fused) k_mdot<T><<<vg, TPB, 0, st>>>(V, vstride, nvec, W, ld, n, live2, part, G, nullptr);
    k_dot_reduce<<<rb, 256, 0, st>>>(part, G, nvec, k, live2, hp, ldp, H, ldh, hoff, 1);
    k_maxpy<T><<<vg, TPB, 0, st>>>(V, vstride, nvec, W, ld, n, hp, ldp, 1.0, live2, npart, G);
    ECT_CHECK_LAUNCH();
}

// The right-hand sides of a solve fall into groups, each with its own matrix
// (one group for a plain solve; one per frequency for a frequency sweep).
// The Krylov kernels treat all right-hand sides together; the operator and
// the preconditioner are applied group by group.
struct Group {
    int which, r0, k;
    int rhs_r0;  // first right-hand side of the group in the caller's rhs array
};
using Groups = std::vector<Group>;

inline const int* goff(const int* a, const Group& g) { return a ? a + g.r0 : nullptr; }

void g_precond_f32(ect_ctx* c, const Groups& G, const float2* r, float2* z, int64_t ld, int tile, const int* act) {
    for (const Group& g : G)
        precond_apply_f32(c, g.which, r + g.r0 * ld, z + g.r0 * ld, g.k, ld, tile, goff(act, g));
}
void g_spmv_f32(ect_ctx* c, const Groups& G, const float2* x, float2* y, int64_t ld, int tile, const int* act) {
    for (const Group& g : G) spmv_f32(c, g.which, x + g.r0 * ld, y + g.r0 * ld, g.k, ld, tile, goff(act, g));
}
void g_spmv_df32(ect_ctx* c, const Groups& G, const float2* x, double2* y, int64_t ld, int tile, const int* act) {
    for (const Group& g : G) spmv_df32(c, g.which, x + g.r0 * ld, y + g.r0 * ld, g.k, ld, tile, goff(act, g));
}
void g_precond_f64(ect_ctx* c, const Groups& G, const double2* r, double2* z, int64_t ld, int tile, const int* act) {
    for (const Group& g : G)
        precond_apply_f64(c, g.which, r + g.r0 * ld, z + g.r0 * ld, g.k, ld, tile, goff(act, g));
}
void g_spmv_f64(ect_ctx* c, const Groups& G, const double2* x, double2* y, int64_t ld, int tile, const int* act) {
    for (const Group& g : G) spmv_f64(c, g.which, true, x + g.r0 * ld, y + g.r0 * ld, g.k, ld, tile, goff(act, g));
}

// inner FP32 GMRES: z (FP64, Z_j) ~= S^-1 v (FP64, V_j), fixed mi iterations
void inner_solve(ect_ctx* c, Workspace* w, const Groups& G, const double2* v, double2* z, int rhs_tile) {
    cudaStream_t st = c->stream;
    const int k = w->k, mi = w->mi;
    const int64_t n = w->n, ld = n, vs = n * k;
    float2* V32 = w->V32.as<float2>();
    float2* U32 = w->U32.as<float2>();
    float2* Z32 = w->Z32.as<float2>();
    const int* live = w->live.as<int>();
    int* live_i = w->live_i.as<int>();
    k_inner_g0<<<grid_for(k, 128), 128, 0, st>>>(live, k, mi, w->gi.as<double2>(), live_i, w->nit_i.as<int>());
    k_d2f<<<dim3(ew_blocks(n, k), k), TPB, 0, st>>>(v, V32, ld, n, live);
    for (int j = 0; j < mi; ++j) {
        float2* Vj = V32 + (int64_t)j * vs;
        float2* Vn = V32 + (int64_t)(j + 1) * vs;
        float2* Zj = Z32 + (int64_t)j * vs;
        g_precond_f32(c, G, Vj, Zj, ld, rhs_tile, live_i);
        g_spmv_f32(c, G, Zj, Vn, ld, rhs_tile, live_i);
        cgs2_step<float>(c, w, V32, vs, j, Vn, ld, w->Hi.as<double2>(), mi, live_i, w->inner_one_pass);
        k_arnoldi_finalize<<<grid_for((int64_t)k * 32, 128), 128, 0, st>>>(
            w->npart.as<double>(), w->G, k, j, mi, w->Hi.as<double2>(), w->csi.as<double>(), w->sni.as<double2>(),
            w->gi.as<double2>(), w->target_i.as<double>(), live_i, w->nit_i.as<int>(), w->inv_h.as<double>(),
            w->flags.as<int>());
        k_scale_vec<float><<<dim3(ew_blocks(n, k), k), TPB, 0, st>>>(Vn, Vn, ld, n, w->inv_h.as<double>(), live_i, k);
    }
    k_trisolve<<<grid_for(k, 128), 128, 0, st>>>(w->Hi.as<double2>(), w->gi.as<double2>(), w->nit_i.as<int>(), live,
                                                k, mi, w->yi.as<double2>());
    // z = P^-1 (sum_i y_i V32_i) = sum_i y_i Z32_i with the stored Z32_i = P^-1 V32_i
    // (one combination pass instead of one more preconditioner application)
    k_zero<float><<<dim3(ew_blocks(n, k), k), TPB, 0, st>>>(U32, ld, n, live);
    k_maxpy<float><<<vgrid(w), TPB, 0, st>>>(Z32, vs, mi, U32, ld, n, w->yi.as<double2>(), mi + 1, -1.0, live,
                                              nullptr, w->G);
    k_f2d<<<dim3(ew_blocks(n, k), k), TPB, 0, st>>>(U32, z, ld, n, live);
    ECT_CHECK_LAUNCH();
}

// one restart cycle (capturable): starts from R / rnorm, ends with Y updated,
// R = Bh - S Y and rnorm
void run_cycle(ect_ctx* c, Workspace* w, const Groups& G, int rhs_tile) {
    cudaStream_t st = c->stream;
    const int k = w->k, m = w->m;
    const int64_t n = w->n, ld = n, vs = n * k;
    double2* V = w->V.as<double2>();
    double2* Z = w->Z.as<double2>();
    int* live = w->live.as<int>();
    const int* run = w->run.as<int>();
    k_cycle_g0<<<grid_for(k, 128), 128, 0, st>>>(w->rnorm.as<double>(), run, k, m, w->g.as<double2>(),
                                                 w->invb.as<double>(), live, w->nit.as<int>());
    k_scale_vec<double><<<dim3(ew_blocks(n, k), k), TPB, 0, st>>>(w->R.as<double2>(), V, ld, n, w->invb.as<double>(),
                                                                  run, k);
    for (int j = 0; j < m; ++j) {
        double2* Vj = V + (int64_t)j * vs;
        double2* Vn = V + (int64_t)(j + 1) * vs;
        double2* Zj = Z + (int64_t)j * vs;
        if (w->mode == ECT_MODE_MIXED) {
            // Z_j is the FP32 inner solution (U32) widened: its product with S is formed in
            // double-float arithmetic from the FP32 copy and remainder of S
            inner_solve(c, w, G, Vj, Zj, rhs_tile);
            g_spmv_df32(c, G, w->U32.as<float2>(), Vn, ld, rhs_tile, live);
        } else {
            g_precond_f64(c, G, Vj, Zj, ld, rhs_tile, live);
            g_spmv_f64(c, G, Zj, Vn, ld, rhs_tile, live);
        }
        cgs2_step<double>(c, w, V, vs, j, Vn, ld, w->H.as<double2>(), m, live, w->outer_one_pass);
        k_arnoldi_finalize<<<grid_for((int64_t)k * 32, 128), 128, 0, st>>>(
            w->npart.as<double>(), w->G, k, j, m, w->H.as<double2>(), w->cs.as<double>(), w->sn.as<double2>(),
            w->g.as<double2>(), w->target.as<double>(), live, w->nit.as<int>(), w->inv_h.as<double>(),
            w->flags.as<int>());
        k_scale_vec<double><<<dim3(ew_blocks(n, k), k), TPB, 0, st>>>(Vn, Vn, ld, n, w->inv_h.as<double>(), live, k);
    }
    k_trisolve<<<grid_for(k, 128), 128, 0, st>>>(w->H.as<double2>(), w->g.as<double2>(), w->nit.as<int>(), run, k, m,
                                                w->y.as<double2>());
    k_maxpy<double><<<vgrid(w), TPB, 0, st>>>(Z, vs, m, w->Y.as<double2>(), ld, n, w->y.as<double2>(), m + 1, -1.0,
                                              run, nullptr, w->G);
    g_spmv_f64(c, G, w->Y.as<double2>(), w->R.as<double2>(), ld, rhs_tile, run);
    k_residual<<<vgrid(w), TPB, 0, st>>>(w->Bh.as<double2>(), w->R.as<double2>(), ld, n, run, w->npart.as<double>(),
                                        w->G);
    k_norm_finalize<<<grid_for((int64_t)k * 32, 128), 128, 0, st>>>(w->npart.as<double>(), w->G, k, run, w->rnorm.as<double>());
    ECT_CHECK_LAUNCH();
}

}  // namespace

namespace {

void solve_groups(ect_ctx* c, const Groups& G, const double2* rhs, double2* x, int k, const ect_options& opt,
                  ect_stats* stats) {
    ECT_REQUIRE(k >= 1 && k <= 4096, ECT_ERR_ARG, "k must be in [1, 4096]");
    ECT_REQUIRE(rhs && x, ECT_ERR_ARG, "null rhs or x");
    ECT_REQUIRE(opt.restart >= 1 && opt.restart <= 64, ECT_ERR_ARG, "restart must be in [1, 64]");
    ECT_REQUIRE(opt.tol >= 0.0 && opt.max_iters >= 1, ECT_ERR_ARG, "bad tol or max_iters");
    ECT_REQUIRE(opt.mode == ECT_MODE_F64 || opt.mode == ECT_MODE_MIXED, ECT_ERR_ARG, "bad mode");
    const int mi = opt.mode == ECT_MODE_MIXED ? opt.inner_iters : 0;
    if (opt.mode == ECT_MODE_MIXED) ECT_REQUIRE(mi >= 1 && mi <= 64, ECT_ERR_ARG, "inner_iters must be in [1, 64]");
    for (const Group& g : G) {
        ECT_REQUIRE(which_valid(c, g.which), ECT_ERR_ARG, "bad which");
        Matrix& M = ctx_mat(c, g.which);
        ECT_REQUIRE(M.assembled && M.pc_f64, ECT_ERR_STATE, "assemble and set up the preconditioner first");
        if (opt.mode == ECT_MODE_MIXED)
            ECT_REQUIRE(M.has_f32 && M.pc_f32, ECT_ERR_STATE, "mixed mode needs the FP32 matrix and preconditioner");
    }
    cudaStream_t st = c->stream;
    ECT_REQUIRE(opt.spmm_rows >= -2 && opt.spmm_rows <= 64, ECT_ERR_ARG, "spmm_rows must be -2, -1 or in [0, 64]");
    c->staged_rows = opt.spmm_rows == 0 ? STAGED_ROWS_DEFAULT : opt.spmm_rows;
    if (opt.mode == ECT_MODE_MIXED)
        for (const Group& g : G) staged_prepare(c, g.which);
    ECT_CUDA(cudaEventRecord(c->ev0, st));
    for (const Group& g : G) coarse_scratch(c, g.which, g.k);
    Workspace* w = get_ws(c, k, opt.restart, mi, opt.mode);
    const bool in1 = opt.reorth >= 2, out1 = opt.reorth == 3;
    if (w->selective != (opt.reorth != 0) || w->inner_one_pass != in1 || w->outer_one_pass != out1) {
        for (auto& kv : w->graphs) cudaGraphExecDestroy(kv.second.first);
        w->graphs.clear();
        w->selective = opt.reorth != 0;
        w->inner_one_pass = in1;
        w->outer_one_pass = out1;
    }
    const int64_t n = w->n, ld = n;
    // scaled right-hand side and its norms; Y = 0, R = Bh
    for (const Group& g : G)
        k_diag_scale<<<dim3(ew_blocks(n, g.k), g.k), TPB, 0, st>>>(rhs + g.rhs_r0 * ld, w->Bh.as<double2>() + g.r0 * ld,
                                                                  ctx_mat(c, g.which).t.as<double>(), ld, n);
    k_norm_part<double><<<vgrid(w), TPB, 0, st>>>(w->Bh.as<double2>(), ld, n, nullptr, w->npart.as<double>(), w->G);
    k_norm_finalize<<<grid_for((int64_t)k * 32, 128), 128, 0, st>>>(w->npart.as<double>(), w->G, k, nullptr, w->bnorm.as<double>());
    if (opt.x0) {
        // Y = T^-1 x0, R = Bh - S Y and its norm
        for (const Group& g : G)
            k_diag_unscale<<<dim3(ew_blocks(n, g.k), g.k), TPB, 0, st>>>(x + g.r0 * ld, w->Y.as<double2>() + g.r0 * ld,
                                                                        ctx_mat(c, g.which).t.as<double>(), ld, n);
        const std::vector<int> all(k, 1);
        ECT_CUDA(cudaMemcpyAsync(w->run.p, all.data(), sizeof(int) * k, cudaMemcpyHostToDevice, st));
        g_spmv_f64(c, G, w->Y.as<double2>(), w->R.as<double2>(), ld, opt.rhs_tile, w->run.as<int>());
        k_residual<<<vgrid(w), TPB, 0, st>>>(w->Bh.as<double2>(), w->R.as<double2>(), ld, n, w->run.as<int>(),
                                            w->npart.as<double>(), w->G);
        k_norm_finalize<<<grid_for((int64_t)k * 32, 128), 128, 0, st>>>(w->npart.as<double>(), w->G, k,
                                                                        w->run.as<int>(), w->rnorm.as<double>());
        ECT_CHECK_LAUNCH();
    } else {
        ECT_CUDA(cudaMemsetAsync(w->Y.p, 0, sizeof(double2) * n * k, st));
        ECT_CUDA(cudaMemcpyAsync(w->R.p, w->Bh.p, sizeof(double2) * n * k, cudaMemcpyDeviceToDevice, st));
        ECT_CUDA(cudaMemcpyAsync(w->rnorm.p, w->bnorm.p, sizeof(double) * k, cudaMemcpyDeviceToDevice, st));
    }
    ECT_CUDA(cudaMemsetAsync(w->flags.p, 0, sizeof(int), st));
    std::vector<double> bnorm(k), rnorm(k), target(k), target_i(k, 0.0);
    ECT_CUDA(cudaMemcpyAsync(bnorm.data(), w->bnorm.p, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
    ECT_CUDA(cudaMemcpyAsync(rnorm.data(), w->rnorm.p, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
    ECT_CUDA(cudaStreamSynchronize(st));
    for (int r = 0; r < k; ++r) target[r] = opt.tol * bnorm[r];
    ECT_CUDA(cudaMemcpyAsync(w->target.p, target.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
    if (mi) ECT_CUDA(cudaMemcpyAsync(w->target_i.p, target_i.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
    std::vector<int> run(k), nit(k), iters(k, 0), outer(k, 0);
    const bool graphs = opt.use_graph && st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread;
    auto t_start = std::chrono::steady_clock::now();
    int restarts = 0, status = ECT_OK;
    int64_t launches = 4;  // scaling, norms (outside the cycles)
    while (true) {
        int n_run = 0, total_outer = 0;
        for (int r = 0; r < k; ++r) {
            run[r] = (rnorm[r] > target[r]) && (outer[r] < opt.max_iters) && bnorm[r] > 0.0;
            n_run += run[r];
            total_outer = std::max(total_outer, outer[r]);
        }
        if (n_run == 0) break;
        if (opt.timeout_s > 0.0) {
            double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
            if (el > opt.timeout_s) {
                status = ECT_ERR_TIMEOUT;
                break;
            }
        }
        ECT_CUDA(cudaMemcpyAsync(w->run.p, run.data(), sizeof(int) * k, cudaMemcpyHostToDevice, st));
        if (graphs) {
            auto key = std::make_tuple(G[0].which + 1000 * (int)G.size(), opt.mode, opt.rhs_tile, c->staged_rows,
                                       c->plan_gen);
            auto it = w->graphs.find(key);
            if (it == w->graphs.end()) {
                cudaGraph_t gr;
                ECT_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                try {
                    run_cycle(c, w, G, opt.rhs_tile);
                } catch (...) {
                    cudaStreamEndCapture(st, &gr);
                    throw;
                }
                ECT_CUDA(cudaStreamEndCapture(st, &gr));
                size_t nn = 0;
                ECT_CUDA(cudaGraphGetNodes(gr, nullptr, &nn));
                cudaGraphExec_t ex;
                ECT_CUDA(cudaGraphInstantiate(&ex, gr, 0));
                cudaGraphDestroy(gr);
                it = w->graphs.emplace(key, std::make_pair(ex, nn)).first;
            }
            ECT_CUDA(cudaGraphLaunch(it->second.first, st));
            launches += (int64_t)it->second.second;
        } else {
            run_cycle(c, w, G, opt.rhs_tile);
        }
        ECT_CUDA(cudaMemcpyAsync(rnorm.data(), w->rnorm.p, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        ECT_CUDA(cudaMemcpyAsync(nit.data(), w->nit.p, sizeof(int) * k, cudaMemcpyDeviceToHost, st));
        int h_flags = 0;
        ECT_CUDA(cudaMemcpyAsync(&h_flags, w->flags.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        ECT_CUDA(cudaStreamSynchronize(st));
        ++restarts;
        for (int r = 0; r < k; ++r)
            if (run[r]) {
                outer[r] += nit[r];
                iters[r] += nit[r] * (mi ? mi : 1);
            }
        if (h_flags) {
            status = ECT_ERR_BREAKDOWN;
            break;
        }
        bool stalled = true;
        for (int r = 0; r < k; ++r)
            if (run[r] && nit[r] > 0) stalled = false;
        if (stalled) break;
    }
    launches += 1;
    // x = T y
    for (const Group& g : G)
        k_diag_scale<<<dim3(ew_blocks(n, g.k), g.k), TPB, 0, st>>>(w->Y.as<double2>() + g.r0 * ld, x + g.r0 * ld,
                                                                  ctx_mat(c, g.which).t.as<double>(), ld, n);
    ECT_CHECK_LAUNCH();
    ECT_CUDA(cudaEventRecord(c->ev1, st));
    ECT_CUDA(cudaEventSynchronize(c->ev1));
    float ms = 0.f;
    ECT_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    int conv = 0, maxit = 0, maxout = 0;
    double worst = 0.0;
    for (int r = 0; r < k; ++r) {
        double rel = bnorm[r] > 0.0 ? rnorm[r] / bnorm[r] : 0.0;
        if (rel <= opt.tol) ++conv;
        worst = std::max(worst, rel);
        maxit = std::max(maxit, iters[r]);
        maxout = std::max(maxout, outer[r]);
    }
    if (stats) {
        stats->iters = maxit;
        stats->outer_iters = maxout;
        stats->converged = conv;
        stats->restarts = restarts;
        stats->relres_max = worst;
        stats->ms = ms;
        stats->launches = launches;
    }
    if (opt.mode == ECT_MODE_MIXED && c->staged_rows > 0 && staged_take_error(st))
        throw EctError{ECT_ERR_TIMEOUT, "a bounded wait for a bulk copy expired in the staged SpMM"};
    if (status != ECT_OK) {
        throw EctError{status, status == ECT_ERR_TIMEOUT ? "solve timed out" : "NaN/Inf in the Krylov recurrence"};
    }
    if (conv < k) throw EctError{ECT_ERR_NOT_CONVERGED, "tolerance not reached within max_iters"};
}

}  // namespace

void solve(ect_ctx* c, int which, const double2* rhs, double2* x, int k, const ect_options& opt, ect_stats* stats) {
    ECT_REQUIRE(which_valid(c, which), ECT_ERR_ARG, "bad which");
    solve_groups(c, Groups{Group{which, 0, k, 0}}, rhs, x, k, opt, stats);
}

void solve_sweep(ect_ctx* c, int config, const double2* rhs, double2* x, int k, const ect_options& opt,
                 ect_stats* stats, bool same_rhs) {
    ECT_REQUIRE(config == ECT_VACUUM || config == ECT_DEFECT, ECT_ERR_ARG, "config must be ECT_VACUUM or ECT_DEFECT");
    const int F = (int)c->sweep_omega.size();
    ECT_REQUIRE(F >= 1, ECT_ERR_STATE, "no frequency sweep assembled (ect_assemble_sweep)");
    ECT_REQUIRE(k >= 1 && (int64_t)k * F <= 4096, ECT_ERR_ARG, "k per frequency must be >= 1 and k * F <= 4096");
    Groups G;
    for (int f = 0; f < F; ++f) G.push_back(Group{2 + 2 * f + config, f * k, k, same_rhs ? 0 : f * k});
    solve_groups(c, G, rhs, x, k * F, opt, stats);
}

void cgs2_entry(ect_ctx* c, int precision, const void* V, int j, int64_t n, void* w, double* h, double* beta) {
    ECT_REQUIRE(V && w && h && beta, ECT_ERR_ARG, "null argument");
    ECT_REQUIRE(j >= 1 && j <= 64 && n >= 1, ECT_ERR_ARG, "need 1 <= j <= 64 and n >= 1");
    ECT_REQUIRE(precision == ECT_F64 || precision == ECT_F32, ECT_ERR_ARG, "bad precision");
    Workspace tmp;
    tmp.k = 1;
    tmp.m = j;
    tmp.mi = 0;
    tmp.n = n;
    tmp.G = pick_G(n, 1);
    tmp.part.alloc(sizeof(double2) * (j + 1) * tmp.G);
    tmp.npart.alloc(sizeof(double) * tmp.G);
    tmp.selective = false;
    tmp.hp.alloc(sizeof(double2) * (j + 1));
    DevBuf H, nrm;
    H.alloc(sizeof(double2) * (j + 1) * j);
    nrm.alloc(sizeof(double));
    cudaStream_t st = c->stream;
    // H column 0 receives the coefficients (layout of column j-1 with m = j: offset (j-1)(j+1))
    if (precision == ECT_F64)
        cgs2_step<double>(c, &tmp, (const double2*)V, n, j - 1, (double2*)w, n, H.as<double2>(), j, nullptr);
    else
        cgs2_step<float>(c, &tmp, (const float2*)V, n, j - 1, (float2*)w, n, H.as<double2>(), j, nullptr);
    k_norm_finalize<<<1, 32, 0, st>>>(tmp.npart.as<double>(), tmp.G, 1, nullptr, nrm.as<double>());
    ECT_CHECK_LAUNCH();
    ECT_CUDA(cudaMemcpyAsync(h, H.as<double2>() + (int64_t)(j - 1) * (j + 1), sizeof(double2) * j,
                             cudaMemcpyDeviceToHost, st));
    ECT_CUDA(cudaMemcpyAsync(beta, nrm.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    ECT_CUDA(cudaStreamSynchronize(st));
}
