// The Delta Z surrogate: a 6 -> 256 x4 -> 256 MLP (SiLU hidden activations,
// linear output) trained and evaluated with tcgen05 tensor-core GEMMs
// (bf16 operands, fp32 accumulation in TMEM) and an Adam optimiser with fp32
// master weights.  It maps deposit parameters to the Delta Z signal along the
// probe path; the solver is its data source and the reference for its error.
//
// Per training step: 5 forward GEMMs (epilogue: bias, SiLU, bf16 copies of
// the activations in the two layouts the backward pass consumes), the loss
// gradient, and per layer dW = dZ^T X and dX = dZ W (epilogue: SiLU'), the
// bias gradients, and Adam, which also rewrites the bf16 weight copies.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "mlp_gemm.cuh"

namespace {

constexpr int NL = 5;
constexpr int IN = 6, IN_PAD = 16, H = 256, OUT = 256;
const int kIn[NL] = {IN, H, H, H, H};
const int kInPad[NL] = {IN_PAD, H, H, H, H};
const int kOut[NL] = {H, H, H, H, OUT};

// pack x [B][6] fp32 -> canonical bf16 (B x 16) and its transpose (16 x B)
__global__ void k_pack_input(const float* __restrict__ x, int B, uint8_t* __restrict__ Xc, uint8_t* __restrict__ XTc) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    for (int k = 0; k < IN_PAD; ++k) {
        const float v = k < IN ? x[(int64_t)b * IN + k] : 0.0f;
        mlpk::put_bf16(Xc, tc05::canon_off(b, k, IN_PAD), v);
        mlpk::put_bf16(XTc, tc05::canon_off(k, b, B), v);
    }
}

// dY = (y - t) / (B D): fp32, canonical (B x D) and transposed canonical; loss partials
__global__ void k_loss_grad(const float* __restrict__ y, const float* __restrict__ t, int B, int D,
                            float* __restrict__ dz, uint8_t* __restrict__ Xc, uint8_t* __restrict__ XTc,
                            double* __restrict__ lpart) {
    __shared__ double sh[8];
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double l = 0.0;
    if (e < (int64_t)B * D) {
        const int b = (int)(e / D), d = (int)(e % D);
        const float r = y[e] - t[e];
        l = 0.5 * (double)r * (double)r;
        const float g = r / (float)((int64_t)B * D);
        dz[e] = g;
        mlpk::put_bf16(Xc, tc05::canon_off(b, d, D), g);
        mlpk::put_bf16(XTc, tc05::canon_off(d, b, B), g);
    }
    l = warp_sum(l);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        lpart[blockIdx.x] = s;
    }
}

// bias gradient, two passes in a fixed order: part[y][n] = sum over the rows of chunk y of
// dz[b][n], then db[n] = sum over y of part[y][n]
constexpr int BIAS_CHUNKS = 64;

__global__ void k_bias_grad_part(const float* __restrict__ dz, int B, int N, float* __restrict__ part) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int rows = (B + BIAS_CHUNKS - 1) / BIAS_CHUNKS;
    const int b0 = blockIdx.y * rows, b1 = min(B, b0 + rows);
    float s = 0.0f;
    for (int b = b0; b < b1; ++b) s += dz[(int64_t)b * N + n];
    part[(int64_t)blockIdx.y * N + n] = s;
}

__global__ void k_bias_grad_sum(const float* __restrict__ part, int N, float* __restrict__ db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.0f;
    for (int y = 0; y < BIAS_CHUNKS; ++y) s += part[(int64_t)y * N + n];
    db[n] = s;
}

// Adam on one layer; rewrites the bf16 weight copies W (out x in_pad) and WT (in_pad x out)
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, int out, int in, int in_pad, int nw, float lr, float b1,
                       float b2, float eps, float c1, float c2, uint8_t* __restrict__ Wc, uint8_t* __restrict__ WTc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (i < nw) {
        const int o = (int)(i / in), k = (int)(i % in);
        mlpk::put_bf16(Wc, tc05::canon_off(o, k, in_pad), pi);
        if (WTc) mlpk::put_bf16(WTc, tc05::canon_off(k, o, out), pi);
    }
}

// bf16 copies of the weights from the fp32 masters (after set_params)
__global__ void k_weights_to_bf16(const float* __restrict__ p, int out, int in, int in_pad, uint8_t* __restrict__ Wc,
                                  uint8_t* __restrict__ WTc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)out * in_pad) return;
    const int o = (int)(i / in_pad), k = (int)(i % in_pad);
    const float w = k < in ? p[(int64_t)o * in + k] : 0.0f;
    mlpk::put_bf16(Wc, tc05::canon_off(o, k, in_pad), w);
    if (WTc) mlpk::put_bf16(WTc, tc05::canon_off(k, o, out), w);
}

}  // namespace

struct ect_mlp {
    cudaStream_t stream = nullptr;
    int B = 0;
    std::string err;
    int64_t off[NL + 1];          // parameter offsets (floats): per layer W (out x in) then b (out)
    DevBuf params, grads, m1, m2; // fp32
    DevBuf Wc[NL], WTc[NL];       // bf16 canonical weights (out x in_pad) and transposes (in_pad x out)
    DevBuf Xc[NL], XTc[NL];       // layer inputs, canonical B x in_pad and in_pad x B
    DevBuf Zf[NL];                // pre-activations (fp32, B x out)
    DevBuf Y;                     // output fp32 B x OUT
    DevBuf dZf, dZc, dZTc;        // current dz (fp32, canonical, transposed canonical)
    DevBuf dZf2, dZc2, dZTc2;     // ping-pong
    DevBuf lpart, errflag;
    DevBuf part;                  // split-K partial products of the weight-gradient GEMMs
    DevBuf bpart;                 // bias-gradient partial sums
    int n_sms = 0;
    int t = 0;
};

namespace {

int64_t n_params_of(int l) { return (int64_t)kOut[l] * kIn[l] + kOut[l]; }

void gemm(ect_mlp* m, const uint8_t* A, const uint8_t* Bm, int M, int N, int K, int mode, const float* bias,
          const float* zprev, float* Zf, float* Yf, uint8_t* Xc, uint8_t* XTc) {
    using namespace mlpk;
    ECT_REQUIRE(M % 128 == 0 && M > 0 && N % 16 == 0 && N >= 16 && N <= 256 && K % 16 == 0 && K >= 16 &&
                    (K <= KCH_MAX || K % KCH_MAX == 0),
                ECT_ERR_ARG, "unsupported GEMM shape");
    GemmArgs g{};
    g.A = A;
    g.B = Bm;
    g.M = M;
    g.N = N;
    g.K = K;
    g.mode = mode;
    g.bias = bias;
    g.zprev = zprev;
    g.Zf = Zf;
    g.Yf = Yf;
    g.Xc = Xc;
    g.XTc = XTc;
    g.err = m->errflag.as<int>();
    g.kch = K < KCH_MAX ? K : KCH_MAX;
    const int nch = K / g.kch, mtiles = M / 128;
    g.resident = (mode != BWD_DW && (uint32_t)N * K * 2 <= RESIDENT_B_MAX) ? 1 : 0;
    ECT_REQUIRE(g.resident || mode == BWD_DW, ECT_ERR_ARG, "weights too large for the resident-B GEMM");
    g.nsplit = 1;
    g.ksplit = nch;
    if (mode == BWD_DW) {  // K (the batch) split so that the items fill the SMs
        const int want = std::max(1, std::min(nch, m->n_sms / mtiles));
        g.ksplit = (nch + want - 1) / want;
        g.nsplit = (nch + g.ksplit - 1) / g.ksplit;
    }
    g.a_bytes = 128u * (uint32_t)g.kch * 2u;
    g.stage_tx = g.a_bytes + (g.resident ? 0u : (uint32_t)N * g.kch * 2u);
    g.stage_bytes = (g.stage_tx + 1023u) / 1024u * 1024u;
    g.b_tx = g.resident ? (uint32_t)N * K * 2u : 0u;
    g.b_bytes = (g.b_tx + 1023u) / 1024u * 1024u;
    const int room = PIPE_SMEM_MAX - (int)g.b_bytes - EPI_BYTES;
    g.stages = std::min(PIPE_MAX_STAGES, room / (int)g.stage_bytes);
    ECT_REQUIRE(g.stages >= 2, ECT_ERR_ARG, "GEMM stages do not fit in shared memory (internal)");
    if (g.nsplit > 1) {
        const size_t need = sizeof(float) * (size_t)g.nsplit * M * N;
        if (m->part.bytes < need) m->part.alloc(need);
        g.part = m->part.as<float>();
    }
    const size_t smem = (size_t)g.b_bytes + (size_t)g.stages * g.stage_bytes + EPI_BYTES;
    ECT_CUDA(cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int items = mtiles * g.nsplit;
    const int grid = std::min(items, m->n_sms);
    k_gemm_tc<<<grid, PIPE_THREADS, smem, m->stream>>>(g);
    ECT_CHECK_LAUNCH();
    if (g.nsplit > 1) {
        const int64_t n4 = (int64_t)M * N / 4;
        k_sum_splits<<<grid_for(n4, 256), 256, 0, m->stream>>>(reinterpret_cast<const float4*>(g.part), g.nsplit, n4,
                                                             reinterpret_cast<float4*>(Yf));
        ECT_CHECK_LAUNCH();
    }
}

// train: keep what the backward pass reads (pre-activations, transposed activations)
void forward(ect_mlp* m, const float* d_x, bool train) {
    const int B = m->B;
    cudaStream_t st = m->stream;
    k_pack_input<<<grid_for(B, 128), 128, 0, st>>>(d_x, B, m->Xc[0].as<uint8_t>(), m->XTc[0].as<uint8_t>());
    ECT_CHECK_LAUNCH();
    const float* P = m->params.as<float>();
    for (int l = 0; l < NL; ++l) {
        const float* bias = P + m->off[l] + (int64_t)kOut[l] * kIn[l];
        if (l < NL - 1)
            gemm(m, m->Xc[l].as<uint8_t>(), m->Wc[l].as<uint8_t>(), B, kOut[l], kInPad[l],
                 train ? mlpk::FWD_HIDDEN : mlpk::FWD_INFER, bias, nullptr, m->Zf[l].as<float>(), nullptr,
                 m->Xc[l + 1].as<uint8_t>(), m->XTc[l + 1].as<uint8_t>());
        else
            gemm(m, m->Xc[l].as<uint8_t>(), m->Wc[l].as<uint8_t>(), B, kOut[l], kInPad[l], mlpk::FWD_OUT, bias,
                 nullptr, nullptr, m->Y.as<float>(), nullptr, nullptr);
    }
}

// forward + loss + backward: fills m->grads; returns loss partial count
int backward(ect_mlp* m, const float* d_x, const float* d_t) {
    const int B = m->B;
    cudaStream_t st = m->stream;
    forward(m, d_x, true);
    const int64_t nout = (int64_t)B * OUT;
    const int lb = (int)grid_for(nout, 256);
    k_loss_grad<<<lb, 256, 0, st>>>(m->Y.as<float>(), d_t, B, OUT, m->dZf.as<float>(), m->dZc.as<uint8_t>(),
                                    m->dZTc.as<uint8_t>(), m->lpart.as<double>());
    ECT_CHECK_LAUNCH();
    float* G = m->grads.as<float>();
    DevBuf* cur[3] = {&m->dZf, &m->dZc, &m->dZTc};
    DevBuf* nxt[3] = {&m->dZf2, &m->dZc2, &m->dZTc2};
    for (int l = NL - 1; l >= 0; --l) {
        float* gW = G + m->off[l];
        float* gb = gW + (int64_t)kOut[l] * kIn[l];
        // dW (out x in_pad) = dZ^T (out x B) * X^T (in_pad x B)^T; keep the first `in` columns
        if (kInPad[l] == kIn[l]) {
            gemm(m, cur[2]->as<uint8_t>(), m->XTc[l].as<uint8_t>(), kOut[l], kInPad[l], B, mlpk::BWD_DW, nullptr,
                 nullptr, nullptr, gW, nullptr, nullptr);
        } else {
            // padded input layer: GEMM into Y (free now) then compact
            gemm(m, cur[2]->as<uint8_t>(), m->XTc[l].as<uint8_t>(), kOut[l], kInPad[l], B, mlpk::BWD_DW, nullptr,
                 nullptr, nullptr, m->Y.as<float>(), nullptr, nullptr);
            ECT_CUDA(cudaMemcpy2DAsync(gW, sizeof(float) * kIn[l], m->Y.p, sizeof(float) * kInPad[l],
                                       sizeof(float) * kIn[l], kOut[l], cudaMemcpyDeviceToDevice, st));
        }
        k_bias_grad_part<<<dim3((unsigned)grid_for(kOut[l], 128), BIAS_CHUNKS), 128, 0, st>>>(
            cur[0]->as<float>(), B, kOut[l], m->bpart.as<float>());
        ECT_CHECK_LAUNCH();
        k_bias_grad_sum<<<grid_for(kOut[l], 128), 128, 0, st>>>(m->bpart.as<float>(), kOut[l], gb);
        ECT_CHECK_LAUNCH();
        if (l > 0) {
            // dX (B x in) = dZ (B x out) * W (out x in) -> dz_{l-1} = dX * silu'(Z_{l-1})
            gemm(m, cur[1]->as<uint8_t>(), m->WTc[l].as<uint8_t>(), B, kIn[l], kOut[l], mlpk::BWD_DX, nullptr,
                 m->Zf[l - 1].as<float>(), nxt[0]->as<float>(), nullptr, nxt[1]->as<uint8_t>(),
                 nxt[2]->as<uint8_t>());
            std::swap(cur[0], nxt[0]);
            std::swap(cur[1], nxt[1]);
            std::swap(cur[2], nxt[2]);
        }
    }
    return lb;
}

double read_loss(ect_mlp* m, int nparts) {
    std::vector<double> h(nparts);
    ECT_CUDA(cudaMemcpyAsync(h.data(), m->lpart.p, sizeof(double) * nparts, cudaMemcpyDeviceToHost, m->stream));
    int e = 0;
    ECT_CUDA(cudaMemcpyAsync(&e, m->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    ECT_CUDA(cudaStreamSynchronize(m->stream));
    ECT_REQUIRE(!e, ECT_ERR_TIMEOUT, "a tensor-core GEMM wait expired");
    double s = 0.0;
    for (double v : h) s += v;
    return s / ((double)m->B * OUT);
}

void check_err(ect_mlp* m) {
    int e = 0;
    ECT_CUDA(cudaMemcpyAsync(&e, m->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    ECT_CUDA(cudaStreamSynchronize(m->stream));
    ECT_REQUIRE(!e, ECT_ERR_TIMEOUT, "a tensor-core GEMM wait expired");
}

thread_local std::string g_mlp_err = "no error";

template <typename F>
int mguard(ect_mlp* m, F&& f) {
    try {
        f();
        if (m) m->err.clear();
        return ECT_OK;
    } catch (const EctError& e) {
        (m ? m->err : g_mlp_err) = e.msg;
        return e.code;
    } catch (...) {
        (m ? m->err : g_mlp_err) = "unknown error";
        return ECT_ERR_ARG;
    }
}

}  // namespace

extern "C" {

int ect_mlp_num_params(void) {
    int64_t s = 0;
    for (int l = 0; l < NL; ++l) s += n_params_of(l);
    return (int)s;
}

int ect_mlp_create(ect_mlp** out, void* stream, int batch) {
    return mguard(nullptr, [&] {
        ECT_REQUIRE(out, ECT_ERR_ARG, "null out");
        ECT_REQUIRE(batch >= 128 && batch % 128 == 0 && (batch <= 256 || batch % 256 == 0) && batch <= 65536,
                    ECT_ERR_ARG, "batch must be a multiple of 128 (and of 256 above 256)");
        *out = nullptr;
        ect_mlp* m = new ect_mlp();
        try {
            m->stream = (cudaStream_t)stream;
            m->B = batch;
            m->off[0] = 0;
            for (int l = 0; l < NL; ++l) m->off[l + 1] = m->off[l] + n_params_of(l);
            const int64_t np = m->off[NL];
            for (DevBuf* b : {&m->params, &m->grads, &m->m1, &m->m2}) {
                b->alloc(sizeof(float) * np);
                ECT_CUDA(cudaMemsetAsync(b->p, 0, b->bytes, m->stream));
            }
            for (int l = 0; l < NL; ++l) {
                m->Wc[l].alloc((size_t)2 * kOut[l] * kInPad[l]);
                if (l > 0) m->WTc[l].alloc((size_t)2 * kOut[l] * kInPad[l]);
                m->Xc[l].alloc((size_t)2 * batch * kInPad[l]);
                m->XTc[l].alloc((size_t)2 * batch * kInPad[l]);
                m->Zf[l].alloc(sizeof(float) * batch * kOut[l]);
                ECT_CUDA(cudaMemsetAsync(m->Wc[l].p, 0, m->Wc[l].bytes, m->stream));
            }
            m->Y.alloc(sizeof(float) * (size_t)batch * OUT);
            for (DevBuf* b : {&m->dZf, &m->dZf2}) b->alloc(sizeof(float) * (size_t)batch * H);
            for (DevBuf* b : {&m->dZc, &m->dZTc, &m->dZc2, &m->dZTc2}) b->alloc((size_t)2 * batch * H);
            m->lpart.alloc(sizeof(double) * grid_for((int64_t)batch * OUT, 256));
            m->errflag.alloc(sizeof(int));
            m->bpart.alloc(sizeof(float) * BIAS_CHUNKS * std::max(H, OUT));
            int dev = 0;
            ECT_CUDA(cudaGetDevice(&dev));
            ECT_CUDA(cudaDeviceGetAttribute(&m->n_sms, cudaDevAttrMultiProcessorCount, dev));
            ECT_CUDA(cudaMemsetAsync(m->errflag.p, 0, sizeof(int), m->stream));
            ECT_CUDA(cudaStreamSynchronize(m->stream));
        } catch (...) {
            delete m;
            throw;
        }
        *out = m;
    });
}

void ect_mlp_destroy(ect_mlp* m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    delete m;
}

const char* ect_mlp_last_error(const ect_mlp* m) {
    if (!m) return g_mlp_err.c_str();
    return m->err.empty() ? "no error" : m->err.c_str();
}

int ect_mlp_set_params(ect_mlp* m, const float* h_params) {
    if (!m) return ECT_ERR_ARG;
    return mguard(m, [&] {
        ECT_REQUIRE(h_params, ECT_ERR_ARG, "null params");
        ECT_CUDA(cudaMemcpyAsync(m->params.p, h_params, m->params.bytes, cudaMemcpyHostToDevice, m->stream));
        ECT_CUDA(cudaMemsetAsync(m->m1.p, 0, m->m1.bytes, m->stream));
        ECT_CUDA(cudaMemsetAsync(m->m2.p, 0, m->m2.bytes, m->stream));
        m->t = 0;
        for (int l = 0; l < NL; ++l) {
            k_weights_to_bf16<<<grid_for((int64_t)kOut[l] * kInPad[l], 256), 256, 0, m->stream>>>(
                m->params.as<float>() + m->off[l], kOut[l], kIn[l], kInPad[l], m->Wc[l].as<uint8_t>(),
                l > 0 ? m->WTc[l].as<uint8_t>() : nullptr);
            ECT_CHECK_LAUNCH();
        }
        ECT_CUDA(cudaStreamSynchronize(m->stream));
    });
}

int ect_mlp_get_params(ect_mlp* m, float* h_params) {
    if (!m) return ECT_ERR_ARG;
    return mguard(m, [&] {
        ECT_REQUIRE(h_params, ECT_ERR_ARG, "null params");
        ECT_CUDA(cudaMemcpyAsync(h_params, m->params.p, m->params.bytes, cudaMemcpyDeviceToHost, m->stream));
        ECT_CUDA(cudaStreamSynchronize(m->stream));
    });
}

int ect_mlp_forward(ect_mlp* m, const float* d_x, float* d_y) {
    if (!m) return ECT_ERR_ARG;
    return mguard(m, [&] {
        ECT_REQUIRE(d_x && d_y, ECT_ERR_ARG, "null x or y");
        forward(m, d_x, false);
        ECT_CUDA(cudaMemcpyAsync(d_y, m->Y.p, sizeof(float) * (size_t)m->B * OUT, cudaMemcpyDeviceToDevice,
                                 m->stream));
        check_err(m);
    });
}

int ect_mlp_gradients(ect_mlp* m, const float* d_x, const float* d_t, float* h_grads, double* h_loss) {
    if (!m) return ECT_ERR_ARG;
    return mguard(m, [&] {
        ECT_REQUIRE(d_x && d_t, ECT_ERR_ARG, "null x or t");
        const int nl = backward(m, d_x, d_t);
        if (h_grads)
            ECT_CUDA(cudaMemcpyAsync(h_grads, m->grads.p, m->grads.bytes, cudaMemcpyDeviceToHost, m->stream));
        const double l = read_loss(m, nl);
        if (h_loss) *h_loss = l;
    });
}

int ect_mlp_train_step(ect_mlp* m, const float* d_x, const float* d_t, float lr, double* h_loss) {
    if (!m) return ECT_ERR_ARG;
    return mguard(m, [&] {
        ECT_REQUIRE(d_x && d_t && lr > 0.0f, ECT_ERR_ARG, "bad train_step arguments");
        const int nl = backward(m, d_x, d_t);
        m->t += 1;
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        const float c1 = 1.0f - powf(b1, (float)m->t), c2 = 1.0f - powf(b2, (float)m->t);
        for (int l = 0; l < NL; ++l) {
            const int64_t n = n_params_of(l), o = m->off[l];
            k_adam<<<grid_for(n, 256), 256, 0, m->stream>>>(
                m->params.as<float>() + o, m->grads.as<float>() + o, m->m1.as<float>() + o, m->m2.as<float>() + o, n,
                kOut[l], kIn[l], kInPad[l], kOut[l] * kIn[l], lr, b1, b2, eps, c1, c2, m->Wc[l].as<uint8_t>(),
                l > 0 ? m->WTc[l].as<uint8_t>() : nullptr);
            ECT_CHECK_LAUNCH();
        }
        if (h_loss) *h_loss = read_loss(m, nl);
    });
}

}  // extern "C"
