// Training samples of the learned scatter surrogate, drawn from a model:
// (event, voxel, line) triples with the network inputs and the exact
// single-scatter sum S_w of the model's path tables (Eq. s_p with n = 1,
// summed over the scatter points, times the detector response) as target.
#include "lmmew_internal.cuh"

namespace lmmew {
namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct SampleParams {
    const float* tab;
    const float* cs;
    const int* q_pix;
    const float* g8;
    const uint16_t* angle;
    const uint16_t* bin;
    const float* energy;
    int64_t n_ev;
    int64_t n;
    uint64_t seed;
    int n_img, A, B, W, nq, nqt, np, npc;
    float h, bin_w;
    float mu_line[LMMEW_MAX_LINES];
    float e_line[LMMEW_MAX_LINES];
    const float* rho;
    float* x;
    float* t;
    int* status;
};

__global__ void k_sample(const SampleParams P) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const uint64_t r0 = mix64(P.seed ^ mix64(3 * (uint64_t)i));
    const uint64_t r1 = mix64(r0);
    const uint64_t r2 = mix64(r1);
    const int64_t e = (int64_t)(r0 % (uint64_t)P.n_ev);
    const int q = (int)(r1 % (uint64_t)P.nq);
    const int w = (int)(r2 % (uint64_t)P.W);
    const int a = P.angle[e], b = P.bin[e];
    const float eh = P.energy[e];
    float* xo = P.x + i * kSurrogateIn;
    if (a >= P.A || b >= P.B || !isfinite(eh)) {
        atomicOr(P.status, kStatusOutOfRange);
        for (int k = 0; k < kSurrogateIn; ++k) xo[k] = 0.f;
        P.t[i] = 0.f;
        return;
    }
    const int pix = P.q_pix[q];
    const float xq = ((pix % P.n_img) + 0.5f - 0.5f * P.n_img) * P.h;
    const float yq = ((pix / P.n_img) + 0.5f - 0.5f * P.n_img) * P.h;
    float ca, sa;
    sincosf(6.283185307179586f * a / P.A, &sa, &ca);
    const float ub = -0.5f * P.B * P.bin_w + (b + 0.5f) * P.bin_w;
    float f[kSurrogateIn];
    surrogate_features(xq, yq, ca, sa, ub, eh, w, P.e_line[w], P.mu_line[w],
                       P.g8 + ((size_t)a * P.nq + q) * 8, P.rho, P.n_img, P.h, f);
    for (int k = 0; k < kSurrogateIn; ++k) xo[k] = f[k];
    // exact single-scatter sum for this line from the FP32 path tables
    const int qt = q / kQT, ql = q % kQT;
    const size_t blk = (size_t)3 * P.W * kQT * kPC;
    double s = 0.0;
    for (int r = 0; r < P.np; ++r) {
        const int pc = r / kPC, sl = r % kPC;
        const float c = P.cs[(((size_t)a * P.npc + pc) * P.B + b) * kCPad + sl];
        if (c == 0.f) continue;
        const float* tb = P.tab + (((size_t)a * P.nqt + qt) * P.npc + pc) * blk;
        // square-root form: alpha s(P) g(e_hat; E') = 2^-(d^2 + nlh), d = sr e_hat + m
        const float nlh = tb[((0 * P.W + w) * kQT + ql) * kPC + sl];
        const float sr = tb[((1 * P.W + w) * kQT + ql) * kPC + sl];
        const float mm = tb[((2 * P.W + w) * kQT + ql) * kPC + sl];
        const double d = (double)sr * eh + mm;
        s += (double)c * exp2(-(d * d + (double)nlh));
    }
    P.t[i] = (float)log(s + (double)kSurrogateEps);
}

}  // namespace
}  // namespace lmmew

using namespace lmmew;

extern "C" int lm_surrogate_sample(lm_handle* h, const lm_events* ev, int64_t n, uint64_t seed,
                                   float* x_out, float* target_out, lm_stream stream) {
    if (!h || !ev || !x_out || !target_out || n < 0)
        return set_error(LMMEW_ERR_INVALID_ARG, "bad argument");
    if (ev->n <= 0 || !ev->angle || !ev->bin || !ev->energy_keV)
        return set_error(LMMEW_ERR_INVALID_ARG, "need a non-empty event list");
    const ModelConst& m = h->mc;
    if (m.W > 3) return set_error(LMMEW_ERR_NOT_IMPLEMENTED, "the surrogate covers up to 3 lines");
    if (m.nq <= 0 || m.W <= 0) return set_error(LMMEW_ERR_INVALID_ARG, "the model has no voxels");
    if (n == 0) return LMMEW_OK;
    if (h->tab_slots && m.np > 0)
        return set_error(LMMEW_ERR_NOT_IMPLEMENTED,
                         "sampling exact targets reads every angle's path tables; make them "
                         "resident first (lm_set_table_streaming(h, 0))");
    cudaStream_t st = (cudaStream_t)stream;
    SampleParams P;
    P.tab = h->d_tab;
    P.cs = h->d_cs;
    P.q_pix = h->d_q_pix;
    P.g8 = h->d_g8;
    P.angle = ev->angle;
    P.bin = ev->bin;
    P.energy = ev->energy_keV;
    P.n_ev = ev->n;
    P.n = n;
    P.seed = seed;
    P.n_img = m.n;
    P.A = m.A;
    P.B = m.B;
    P.W = m.W;
    P.nq = m.nq;
    P.nqt = m.nqt;
    P.np = m.np;
    P.npc = m.npc;
    P.h = (float)m.h;
    P.bin_w = (float)m.bin_w;
    for (int w = 0; w < LMMEW_MAX_LINES; ++w) {
        P.mu_line[w] = (float)h->mu_line[w];
        P.e_line[w] = (float)m.line_e[w];
    }
    P.rho = h->d_rho;
    P.x = x_out;
    P.t = target_out;
    P.status = h->d_status;
    k_sample<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    int status = 0;
    LMMEW_CUDA(cudaMemcpyAsync(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    LMMEW_CUDA(cudaStreamSynchronize(st));
    if (status & kStatusOutOfRange) {
        LMMEW_CUDA(cudaMemset(h->d_status, 0, sizeof(int)));
        return set_error(LMMEW_ERR_OUT_OF_RANGE, "an event is outside the model");
    }
    return LMMEW_OK;
}

extern "C" int lm_set_coarse_stride(lm_handle* h, int stride) {
    if (!h) return set_error(LMMEW_ERR_INVALID_ARG, "handle is NULL");
    if (stride < 2 || stride > 4) return set_error(LMMEW_ERR_INVALID_ARG, "stride must be 2, 3 or 4");
    if (stride == h->coarse_stride) return LMMEW_OK;
    // the node tables of the old spacing go; the coarse form rebuilds them
    cudaFree(h->d_node_q);
    cudaFree(h->d_interp_node);
    cudaFree(h->d_interp_w);
    h->d_node_q = nullptr;
    h->d_interp_node = nullptr;
    h->d_interp_w = nullptr;
    h->n_nodes = 0;
    h->coarse_stride = stride;
    if (h->scatter_model == LMMEW_SCATTER_SURROGATE_COARSE) return build_coarse_nodes(h);
    return LMMEW_OK;
}

extern "C" int lm_set_scatter_model(lm_handle* h, int model, const lm_surrogate* s) {
    if (!h) return set_error(LMMEW_ERR_INVALID_ARG, "handle is NULL");
    if (model < 0 || model > 3) return set_error(LMMEW_ERR_INVALID_ARG, "unknown scatter model");
    const bool learned = model == LMMEW_SCATTER_SURROGATE || model == LMMEW_SCATTER_SURROGATE_COARSE;
    if (learned) {
        if (!s) return set_error(LMMEW_ERR_INVALID_ARG, "surrogate is NULL");
        if (h->mc.W > 3)
            return set_error(LMMEW_ERR_NOT_IMPLEMENTED, "the surrogate covers up to 3 lines");
    }
    if (model == LMMEW_SCATTER_SURROGATE_COARSE) {
        const int rc = build_coarse_nodes(h);
        if (rc != LMMEW_OK) return rc;
    }
    h->scatter_model = model;
    h->surrogate = learned ? s : nullptr;
    return LMMEW_OK;
}
