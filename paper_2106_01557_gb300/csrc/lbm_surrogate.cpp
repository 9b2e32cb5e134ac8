// Host runtime of the learned surrogate: parameters (FP32 master copies,
// Adam moments, BF16 forward and flipped copies), activation buffers, the
// forward and backward passes built from the BF16 tensor-core kernels of
// lbm_conv_tc.cu (tcgen05: convolutions, 64 -> 64 weight gradients) or
// lbm_conv.cu (mma.sync; the other weight gradients and the elementwise
// kernels), and the rollout with LB fallback.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_conv.h"
#include "lbm_internal.h"

using namespace lbm;

namespace {

int sfail(int code, const std::string& m) { return lbm_internal_fail(code, m.c_str()); }

#define SCK(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return sfail(LBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct Layer {
    int cin, cout;            // padded channel counts (16 or C)
    int cin_real, cout_real;  // 4 or C
    float* w = nullptr;       // FP32 master [9][cout][cin]
    float* b = nullptr;       // [cout]
    float* gw = nullptr;
    float* gb = nullptr;
    float* mw = nullptr;
    float* vw = nullptr;
    float* mb = nullptr;
    float* vb = nullptr;
    __nv_bfloat16* w16 = nullptr;    // forward copy
    __nv_bfloat16* wflip = nullptr;  // [9][cin][cout], taps reversed: input gradient
    int nw() const { return 9 * cin * cout; }
};

}  // namespace

struct lbm_surrogate {
    lbm_surrogate_config cfg;
    NormConsts nc;
    std::vector<Layer> layers;  // lift, (b1, b2) x B, proj
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sms = 0;
    long long cap = 0;           // pixels the activation buffers hold
    __nv_bfloat16* x16 = nullptr;  // [P][16]
    float* x32 = nullptr;          // [P][4]
    float* t32 = nullptr;          // [P][4] targets
    float* y32 = nullptr;          // [P][16]
    __nv_bfloat16* dy16 = nullptr; // [P][16]
    std::vector<__nv_bfloat16*> h;   // B + 1 activations [P][C]
    std::vector<__nv_bfloat16*> z1;  // B activations
    __nv_bfloat16* g0 = nullptr;     // gradient buffers [P][C]
    __nv_bfloat16* g1 = nullptr;
    __nv_bfloat16* g2 = nullptr;
    double* d_loss = nullptr;
    unsigned long long* d_cnt = nullptr;  // field checks (4 counts)
    double* d_msum = nullptr;        // mass-layer sums, 2 per image
    double* d_mpart = nullptr;       // their per-block partials (2 MASS_BLOCKS per image)
    double* d_lpart = nullptr;       // loss partials (MSE_BLOCKS)
    float* gpart = nullptr;          // weight- and bias-gradient partials
    int msum_cap = 0;
    int* d_status = nullptr;         // bit 0: a tensor-core wait ran out of time
    double* fields = nullptr;        // 4 planes of the rollout case (device)
    double* pred = nullptr;
    double* ver = nullptr;           // the verified state's fields
    unsigned long long* d_chg = nullptr;  // field change of a verification (4 maxima)
    void* snapshot = nullptr;
    size_t snapshot_bytes = 0;
    long long step_count = 0;        // Adam steps
};

static void s_free(void* p) {
    if (p) cudaFree(p);
}

static void release_acts(lbm_surrogate* s) {
    s_free(s->x16); s_free(s->x32); s_free(s->t32); s_free(s->y32); s_free(s->dy16);
    for (auto* p : s->h) s_free(p);
    for (auto* p : s->z1) s_free(p);
    s->h.clear();
    s->z1.clear();
    s_free(s->g0); s_free(s->g1); s_free(s->g2);
    s->x16 = nullptr; s->x32 = s->t32 = s->y32 = nullptr; s->dy16 = s->g0 = s->g1 = s->g2 = nullptr;
    s->cap = 0;
}

static int ensure_acts(lbm_surrogate* s, long long P, bool train) {
    const bool need_train = train && s->z1.size() < (size_t)s->cfg.blocks;
    if (P <= s->cap && !need_train) return LBM_OK;
    SCK(cudaStreamSynchronize(s->stream));
    release_acts(s);
    const int C = s->cfg.channels;
    const size_t a = (size_t)P * C * sizeof(__nv_bfloat16);
    bool ok = cudaMalloc(&s->x16, (size_t)P * 16 * 2) == cudaSuccess && cudaMalloc(&s->x32, (size_t)P * 4 * 4) == cudaSuccess &&
              cudaMalloc(&s->t32, (size_t)P * 4 * 4) == cudaSuccess && cudaMalloc(&s->y32, (size_t)P * 16 * 4) == cudaSuccess &&
              cudaMalloc(&s->dy16, (size_t)P * 16 * 2) == cudaSuccess;
    const int nh = train ? s->cfg.blocks + 1 : 2;
    for (int i = 0; ok && i < nh; ++i) {
        __nv_bfloat16* p = nullptr;
        ok = cudaMalloc(&p, a) == cudaSuccess;
        s->h.push_back(p);
    }
    const int nz = train ? s->cfg.blocks : 1;
    for (int i = 0; ok && i < nz; ++i) {
        __nv_bfloat16* p = nullptr;
        ok = cudaMalloc(&p, a) == cudaSuccess;
        s->z1.push_back(p);
    }
    if (ok && train)
        ok = cudaMalloc(&s->g0, a) == cudaSuccess && cudaMalloc(&s->g1, a) == cudaSuccess &&
             cudaMalloc(&s->g2, a) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        release_acts(s);
        return sfail(LBM_ERR_OOM, "surrogate activation allocation failed");
    }
    s->cap = P;
    return LBM_OK;
}

static ConvArgs cargs(const __nv_bfloat16* in, const __nv_bfloat16* w, const float* b, int N, int H, int W, int relu) {
    ConvArgs a;
    std::memset(&a, 0, sizeof a);
    a.in = in;
    a.w = w;
    a.bias = b;
    a.N = N;
    a.H = H;
    a.W = W;
    a.in_relu = relu;
    return a;
}

// 3x3 convolution on the configured path
static int conv(lbm_surrogate* s, int cin, int cout, const ConvArgs& a) {
    if (s->cfg.conv_path == 0) {
        SCK(launch_conv_tc(cin, cout, a, s->stream, s->sms, s->d_status));
    } else {
        SCK(launch_conv(cin, cout, a, s->stream, s->sms));
    }
    return LBM_OK;
}

// weight gradient: the 64 -> 64 layers on tcgen05 with the tensor-core path
static int wgrad(lbm_surrogate* s, int cin, int cout, const __nv_bfloat16* in, const __nv_bfloat16* dout, int N,
                 int H, int W, int relu, float* gw) {
    if (s->cfg.conv_path == 0 && cin == 64 && cout == 64) {
        SCK(launch_wgrad_tc(cin, cout, in, dout, N, H, W, relu, gw, s->gpart, s->stream, s->sms, s->d_status));
    } else {
        SCK(launch_wgrad(cin, cout, in, dout, N, H, W, relu, gw, s->gpart, s->stream, s->sms));
    }
    return LBM_OK;
}

#define WGRAD(cin, cout, in, dout, relu, gw)                          \
    do {                                                              \
        int rc_ = wgrad(s, cin, cout, in, dout, N, H, W, relu, gw);   \
        if (rc_) return rc_;                                          \
    } while (0)

#define CONV(cin, cout, a)                \
    do {                                  \
        int rc_ = conv(s, cin, cout, a);  \
        if (rc_) return rc_;              \
    } while (0)

// after a stream synchronisation: fail if a tensor-core wait ran out of time
static int check_status(lbm_surrogate* s) {
    int st = 0;
    SCK(cudaMemcpy(&st, s->d_status, sizeof st, cudaMemcpyDeviceToHost));
    if (st) {
        SCK(cudaMemset(s->d_status, 0, sizeof st));
        return sfail(LBM_ERR_CUDA, "a tensor-core completion wait ran out of time");
    }
    return LBM_OK;
}

// forward pass; with train = true every activation is kept for backward
static int run_forward(lbm_surrogate* s, int N, int H, int W, bool train) {
    const int B = s->cfg.blocks, C = s->cfg.channels;
    const Layer& lift = s->layers[0];
    ConvArgs a = cargs(s->x16, lift.w16, lift.b, N, H, W, 0);
    a.out16 = s->h[0];
    CONV(16, C, a);
    for (int b = 0; b < B; ++b) {
        const Layer& L1 = s->layers[1 + 2 * b];
        const Layer& L2 = s->layers[2 + 2 * b];
        __nv_bfloat16* hin = train ? s->h[b] : s->h[b & 1];
        __nv_bfloat16* hout = train ? s->h[b + 1] : s->h[(b + 1) & 1];
        __nv_bfloat16* z = train ? s->z1[b] : s->z1[0];
        a = cargs(hin, L1.w16, L1.b, N, H, W, 1);
        a.out16 = z;
        CONV(C, C, a);
        a = cargs(z, L2.w16, L2.b, N, H, W, 1);
        a.res16 = hin;
        a.out16 = hout;
        CONV(C, C, a);
    }
    const Layer& proj = s->layers.back();
    a = cargs(train ? s->h[B] : s->h[B & 1], proj.w16, proj.b, N, H, W, 1);
    a.res32 = s->x32;
    a.res32_c = 4;
    a.out32 = s->y32;
    CONV(C, 16, a);
    return LBM_OK;
}

static int run_backward(lbm_surrogate* s, int N, int H, int W) {
    const int B = s->cfg.blocks, C = s->cfg.channels;
    const long long P = (long long)N * H * W;
    for (Layer& L : s->layers) {
        SCK(cudaMemsetAsync(L.gw, 0, (size_t)L.nw() * 4, s->stream));
        SCK(cudaMemsetAsync(L.gb, 0, (size_t)L.cout * 4, s->stream));
    }
    // projection: its input is relu(h_B)
    Layer& proj = s->layers.back();
    WGRAD(C, 16, s->h[B], s->dy16, 1, proj.gw);
    SCK(launch_bgrad(s->dy16, P, 16, proj.gb, s->gpart, s->stream));
    ConvArgs a = cargs(s->dy16, proj.wflip, nullptr, N, H, W, 0);
    a.mask = s->h[B];
    a.out16 = s->g0;  // d h_B
    CONV(16, C, a);
    __nv_bfloat16* dh = s->g0;
    __nv_bfloat16* spare = s->g2;
    for (int b = B - 1; b >= 0; --b) {
        Layer& L1 = s->layers[1 + 2 * b];
        Layer& L2 = s->layers[2 + 2 * b];
        // h_{b+1} = h_b + conv2(relu(z1)); d z2 = d h_{b+1}
        WGRAD(C, C, s->z1[b], dh, 1, L2.gw);
        SCK(launch_bgrad(dh, P, C, L2.gb, s->gpart, s->stream));
        a = cargs(dh, L2.wflip, nullptr, N, H, W, 0);
        a.mask = s->z1[b];
        a.out16 = s->g1;  // d z1
        CONV(C, C, a);
        WGRAD(C, C, s->h[b], s->g1, 1, L1.gw);
        SCK(launch_bgrad(s->g1, P, C, L1.gb, s->gpart, s->stream));
        a = cargs(s->g1, L1.wflip, nullptr, N, H, W, 0);
        a.mask = s->h[b];
        a.res16 = dh;
        a.out16 = spare;  // d h_b = d h_{b+1} + conv1^T(d z1) * [h_b > 0]
        CONV(C, C, a);
        std::swap(dh, spare);
    }
    Layer& lift = s->layers[0];
    WGRAD(16, C, s->x16, dh, 0, lift.gw);
    SCK(launch_bgrad(dh, P, C, lift.gb, s->gpart, s->stream));
    return LBM_OK;
}

// the mass-conserving output layer on y32 (with the targets: also the sums
// the projected loss gradient needs)
static int mass_layer(lbm_surrogate* s, int N, long long HW, const float* t32) {
    if (!s->cfg.conserve_mass) return LBM_OK;
    if (N > s->msum_cap) {
        SCK(cudaStreamSynchronize(s->stream));
        s_free(s->d_msum);
        s_free(s->d_mpart);
        s->d_msum = nullptr;
        s->d_mpart = nullptr;
        s->msum_cap = 0;
        SCK(cudaMalloc(&s->d_msum, 2 * (size_t)N * sizeof(double)));
        SCK(cudaMalloc(&s->d_mpart, 2 * (size_t)MASS_BLOCKS * N * sizeof(double)));
        s->msum_cap = N;
    }
    SCK(launch_mass_layer(s->y32, s->x32, t32, N, HW, s->d_msum, s->d_mpart, s->stream));
    return LBM_OK;
}

static int pack_inputs(lbm_surrogate* s, const double* in, long long P, float* x32, __nv_bfloat16* x16) {
    SCK(launch_pack(in, in + P, in + 2 * P, in + 3 * P, P, s->nc, x16, x32, s->stream));
    return LBM_OK;
}

extern "C" {

int lbm_surrogate_create(const lbm_surrogate_config* cfg, lbm_surrogate** out) {
    if (!cfg || !out) return sfail(LBM_ERR_ARG, "null argument");
    *out = nullptr;
    if (cfg->channels != 64) return sfail(LBM_ERR_ARG, "the tensor-core kernels are built for 64 channels");
    if (cfg->blocks < 1 || cfg->blocks > 64) return sfail(LBM_ERR_ARG, "blocks must lie in [1, 64]");
    if (cfg->K < 1) return sfail(LBM_ERR_ARG, "K must be positive");
    if (cfg->conv_path != 0 && cfg->conv_path != 1) return sfail(LBM_ERR_ARG, "conv_path must be 0 (tcgen05) or 1 (mma.sync)");
    for (int c = 0; c < 4; ++c)
        if (!(cfg->norm_scale[c] > 0)) return sfail(LBM_ERR_ARG, "normalisation scales must be positive");
    lbm_surrogate* s = new (std::nothrow) lbm_surrogate();
    if (!s) return sfail(LBM_ERR_OOM, "host allocation failed");
    s->cfg = *cfg;
    for (int c = 0; c < 4; ++c) {
        s->nc.off[c] = cfg->norm_off[c];
        s->nc.scale[c] = cfg->norm_scale[c];
        s->nc.inv_scale[c] = 1.0 / cfg->norm_scale[c];
    }
    cudaError_t e = cudaSetDevice(cfg->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, cfg->device);
    if (e != cudaSuccess) { delete s; return sfail(LBM_ERR_CUDA, cudaGetErrorString(e)); }
    if (cfg->stream) {
        s->stream = static_cast<cudaStream_t>(cfg->stream);
    } else {
        e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete s; return sfail(LBM_ERR_CUDA, cudaGetErrorString(e)); }
        s->own_stream = true;
    }
    const int C = cfg->channels;
    s->layers.push_back({16, C, 4, C});
    for (int b = 0; b < cfg->blocks; ++b) {
        s->layers.push_back({C, C, C, C});
        s->layers.push_back({C, C, C, C});
    }
    s->layers.push_back({C, 16, C, 4});
    bool ok = true;
    for (Layer& L : s->layers) {
        const size_t nw = (size_t)L.nw();
        ok = ok && cudaMalloc(&L.w, nw * 4) == cudaSuccess && cudaMalloc(&L.gw, nw * 4) == cudaSuccess &&
             cudaMalloc(&L.mw, nw * 4) == cudaSuccess && cudaMalloc(&L.vw, nw * 4) == cudaSuccess &&
             cudaMalloc(&L.b, L.cout * 4) == cudaSuccess && cudaMalloc(&L.gb, L.cout * 4) == cudaSuccess &&
             cudaMalloc(&L.mb, L.cout * 4) == cudaSuccess && cudaMalloc(&L.vb, L.cout * 4) == cudaSuccess &&
             cudaMalloc(&L.w16, nw * 2) == cudaSuccess && cudaMalloc(&L.wflip, nw * 2) == cudaSuccess;
        if (ok) {
            cudaMemset(L.w, 0, nw * 4); cudaMemset(L.mw, 0, nw * 4); cudaMemset(L.vw, 0, nw * 4);
            cudaMemset(L.b, 0, L.cout * 4); cudaMemset(L.mb, 0, L.cout * 4); cudaMemset(L.vb, 0, L.cout * 4);
            cudaMemset(L.w16, 0, nw * 2); cudaMemset(L.wflip, 0, nw * 2);
        }
    }
    ok = ok && cudaMalloc(&s->d_loss, sizeof(double)) == cudaSuccess &&
         cudaMalloc(&s->d_lpart, MSE_BLOCKS * sizeof(double)) == cudaSuccess &&
         cudaMalloc(&s->gpart, grad_scratch_floats(s->sms) * sizeof(float)) == cudaSuccess &&
         cudaMalloc(&s->d_cnt, 4 * sizeof(unsigned long long)) == cudaSuccess &&
         cudaMalloc(&s->d_status, sizeof(int)) == cudaSuccess && cudaMemset(s->d_status, 0, sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        lbm_surrogate_destroy(s);
        return sfail(LBM_ERR_OOM, "surrogate parameter allocation failed");
    }
    *out = s;
    return LBM_OK;
}

int64_t lbm_surrogate_num_params(const lbm_surrogate* s) {
    if (!s) return 0;
    int64_t n = 0;
    for (const Layer& L : s->layers) n += 9LL * L.cin_real * L.cout_real + L.cout_real;
    return n;
}

// parameter order <-> padded device layout
static int copy_params(lbm_surrogate* s, float* host, bool to_device, bool grads) {
    size_t off = 0;
    for (Layer& L : s->layers) {
        std::vector<float> wpad((size_t)L.nw()), bpad((size_t)L.cout);
        if (!to_device) {
            SCK(cudaMemcpy(wpad.data(), grads ? L.gw : L.w, wpad.size() * 4, cudaMemcpyDeviceToHost));
            SCK(cudaMemcpy(bpad.data(), grads ? L.gb : L.b, bpad.size() * 4, cudaMemcpyDeviceToHost));
        } else {
            std::fill(wpad.begin(), wpad.end(), 0.f);
            std::fill(bpad.begin(), bpad.end(), 0.f);
        }
        for (int t = 0; t < 9; ++t)
            for (int o = 0; o < L.cout_real; ++o)
                for (int i = 0; i < L.cin_real; ++i) {
                    float& dev = wpad[((size_t)t * L.cout + o) * L.cin + i];
                    float& hv = host[off + ((size_t)t * L.cout_real + o) * L.cin_real + i];
                    if (to_device) dev = hv; else hv = dev;
                }
        off += 9ull * L.cout_real * L.cin_real;
        for (int o = 0; o < L.cout_real; ++o) {
            if (to_device) bpad[o] = host[off + o]; else host[off + o] = bpad[o];
        }
        off += L.cout_real;
        if (to_device) {
            SCK(cudaMemcpy(L.w, wpad.data(), wpad.size() * 4, cudaMemcpyHostToDevice));
            SCK(cudaMemcpy(L.b, bpad.data(), bpad.size() * 4, cudaMemcpyHostToDevice));
            SCK(launch_refresh(L.w, L.cin, L.cout, L.cin_real, L.cout_real, L.w16, L.wflip, s->stream));
        }
    }
    SCK(cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

int lbm_surrogate_set_params(lbm_surrogate* s, const float* params) {
    if (!s || !params) return sfail(LBM_ERR_ARG, "null argument");
    s->step_count = 0;
    for (Layer& L : s->layers) {
        SCK(cudaMemset(L.mw, 0, (size_t)L.nw() * 4));
        SCK(cudaMemset(L.vw, 0, (size_t)L.nw() * 4));
        SCK(cudaMemset(L.mb, 0, (size_t)L.cout * 4));
        SCK(cudaMemset(L.vb, 0, (size_t)L.cout * 4));
    }
    return copy_params(s, const_cast<float*>(params), true, false);
}

int lbm_surrogate_get_params(lbm_surrogate* s, float* params) {
    if (!s || !params) return sfail(LBM_ERR_ARG, "null argument");
    return copy_params(s, params, false, false);
}

static int check_dims(int N, int H, int W) {
    if (N < 1 || H < 1 || W < 16 || W % 16 != 0) return sfail(LBM_ERR_ARG, "need N, H >= 1 and W a multiple of 16");
    return LBM_OK;
}

int lbm_surrogate_forward(lbm_surrogate* s, const double* in, int32_t N, int32_t H, int32_t W, double* out) {
    if (!s || !in || !out) return sfail(LBM_ERR_ARG, "null argument");
    int rc = check_dims(N, H, W);
    if (rc) return rc;
    const long long P = (long long)N * H * W;
    rc = ensure_acts(s, P, false);
    if (rc) return rc;
    rc = pack_inputs(s, in, P, s->x32, s->x16);
    if (rc) return rc;
    rc = run_forward(s, N, H, W, false);
    if (rc) return rc;
    rc = mass_layer(s, N, (long long)H * W, nullptr);
    if (rc) return rc;
    SCK(launch_unpack(s->y32, P, s->nc, out, out + P, out + 2 * P, out + 3 * P, s->stream));
    SCK(cudaStreamSynchronize(s->stream));
    return check_status(s);
}

static int loss_and_backward(lbm_surrogate* s, const double* in, const double* target, int N, int H, int W,
                             double* loss) {
    const long long P = (long long)N * H * W;
    int rc = ensure_acts(s, P, true);
    if (rc) return rc;
    rc = pack_inputs(s, in, P, s->x32, s->x16);
    if (rc) return rc;
    // targets: the normalised 4 fields (the BF16 copy is scratch)
    SCK(launch_pack(target, target + P, target + 2 * P, target + 3 * P, P, s->nc, s->dy16, s->t32, s->stream));
    rc = run_forward(s, N, H, W, true);
    if (rc) return rc;
    rc = mass_layer(s, N, (long long)H * W, s->t32);
    if (rc) return rc;
    SCK(cudaMemsetAsync(s->d_loss, 0, sizeof(double), s->stream));
    SCK(launch_mse(s->y32, s->t32, P, s->dy16, s->d_loss, s->cfg.conserve_mass ? s->d_msum + N : nullptr,
                   (long long)H * W, s->d_lpart, s->stream));
    rc = run_backward(s, N, H, W);
    if (rc) return rc;
    if (loss) {
        SCK(cudaMemcpyAsync(loss, s->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    }
    SCK(cudaStreamSynchronize(s->stream));
    return check_status(s);
}

int lbm_surrogate_loss_grad(lbm_surrogate* s, const double* in, const double* target, int32_t N, int32_t H,
                            int32_t W, double* loss, float* grads) {
    if (!s || !in || !target) return sfail(LBM_ERR_ARG, "null argument");
    int rc = check_dims(N, H, W);
    if (rc) return rc;
    rc = loss_and_backward(s, in, target, N, H, W, loss);
    if (rc) return rc;
    if (grads) return copy_params(s, grads, false, true);
    return LBM_OK;
}

int lbm_surrogate_train_step(lbm_surrogate* s, const double* in, const double* target, int32_t N, int32_t H,
                             int32_t W, double lr, double* loss) {
    if (!s || !in || !target) return sfail(LBM_ERR_ARG, "null argument");
    int rc = check_dims(N, H, W);
    if (rc) return rc;
    if (!(lr > 0)) return sfail(LBM_ERR_ARG, "learning rate must be positive");
    rc = loss_and_backward(s, in, target, N, H, W, loss);
    if (rc) return rc;
    s->step_count += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - std::pow(b1, (float)s->step_count), c2 = 1.f - std::pow(b2, (float)s->step_count);
    for (Layer& L : s->layers) {
        SCK(launch_adam(L.w, L.mw, L.vw, L.gw, L.nw(), (float)lr, b1, b2, eps, c1, c2, s->stream));
        SCK(launch_adam(L.b, L.mb, L.vb, L.gb, L.cout, (float)lr, b1, b2, eps, c1, c2, s->stream));
        SCK(launch_refresh(L.w, L.cin, L.cout, L.cin_real, L.cout_real, L.w16, L.wflip, s->stream));
    }
    SCK(cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

int lbm_surrogate_rollout(lbm_surrogate* s, lbm_handle* h, int32_t njumps, int32_t verify_steps, double drift_tol,
                          double iface_tol, double field_tol, double* stats) {
    if (!s || !h || njumps < 0 || verify_steps < 0 || !(drift_tol > 0) || !(iface_tol > 0) || !(field_tol > 0))
        return sfail(LBM_ERR_ARG, "bad argument");
    double rho_v, rho_l;
    int nx, ny;
    lbm_internal_rho_bounds(h, &rho_v, &rho_l, &nx, &ny);
    int rc = check_dims(1, ny, nx);
    if (rc) return rc;
    const long long P = (long long)nx * ny;
    rc = ensure_acts(s, P, false);
    if (rc) return rc;
    const size_t sb = lbm_internal_state_bytes(h);
    if (!s->fields || s->snapshot_bytes < sb) {
        s_free(s->fields); s_free(s->pred); s_free(s->ver); s_free(s->snapshot); s_free(s->d_chg);
        s->fields = s->pred = s->ver = nullptr; s->snapshot = nullptr; s->d_chg = nullptr;
        if (cudaMalloc(&s->fields, 4 * P * 8) != cudaSuccess || cudaMalloc(&s->pred, 4 * P * 8) != cudaSuccess ||
            cudaMalloc(&s->ver, 4 * P * 8) != cudaSuccess ||
            cudaMalloc(&s->d_chg, 4 * sizeof(unsigned long long)) != cudaSuccess ||
            cudaMalloc(&s->snapshot, sb) != cudaSuccess) {
            cudaGetLastError();
            return sfail(LBM_ERR_OOM, "rollout buffers");
        }
        s->snapshot_bytes = sb;
    }
    double acc = 0, fb = 0, t_sur = 0, t_lb = 0, max_dm = 0, max_de = 0;
    double all_dm = 0, all_de = 0, all_da = 0, n_bad = 0, n_div = 0, all_dr = 0, all_dT = 0;
    const double mid = 0.5 * (rho_v + rho_l);
    // device counts: cnt[0] liquid nodes, cnt[1] unphysical nodes, cnt[2]
    // liquid-vapour edges, cnt[3] nodes whose phase changed from prev
    auto check = [&](const double* f, const double* prev, unsigned long long cnt[4]) {
        SCK(launch_field_check(f, prev, P, nx, mid, s->d_cnt, s->stream));
        SCK(cudaMemcpyAsync(cnt, s->d_cnt, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s->stream));
        SCK(cudaStreamSynchronize(s->stream));
        return LBM_OK;
    };
    cudaStream_t hs = lbm_internal_stream(h);
    using clk = std::chrono::steady_clock;
    auto ms = [](clk::time_point a, clk::time_point b) { return std::chrono::duration<double, std::milli>(b - a).count(); };
    double t_prep = 0, t_net = 0, t_check = 0, t_ver = 0;
    // The state's fields and conservation record are read in one FP32 pass
    // (FP64 sums): the network sees BF16 inputs and the thresholds are far
    // above FP32 rounding. After an accepted jump the read-out that checked it
    // is the next jump's input; a rejected jump keeps the state it read.
    double c0[6], c1[6];
    bool have_state = false;  // s->fields and c0 describe the current state
    for (int j = 0; j < njumps; ++j) {
        unsigned long long n0[4], n1[4];
        const auto tp = clk::now();
        if (!have_state) {
            rc = lbm_internal_read_fast(h, s->fields, c0);
            if (rc) return rc;
        }
        rc = check(s->fields, nullptr, n0);
        if (rc) return rc;
        rc = lbm_internal_snapshot(h, s->snapshot);
        if (rc) return rc;
        const int64_t steps0 = lbm_step_count(h);
        SCK(cudaStreamSynchronize(hs));
        auto t0 = clk::now();
        t_prep += ms(tp, t0);
        rc = lbm_surrogate_forward(s, s->fields, 1, ny, nx, s->pred);
        if (rc) return rc;
        const auto tn = clk::now();
        t_net += ms(t0, tn);
        // an unphysical prediction (non-finite, rho <= 0 or T <= 0) is a rejected jump
        rc = check(s->pred, s->fields, n1);
        if (rc) return rc;
        const bool physical = n1[1] == 0;
        double dm = 0, de = 0, da = 0, dr = 0, dT = 0;
        bool diverged = false;
        auto tv = clk::now();
        if (physical) {
            rc = lbm_internal_set_fields_fast(h, s->pred);
            if (rc) return rc;
            tv = clk::now();
            // the LB re-runs from the surrogate state: a state it cannot
            // advance (non-finite or non-positive density or temperature) is a
            // rejected jump
            if (verify_steps > 0) {
                rc = lbm_step(h, verify_steps);
                if (rc) return rc;
                rc = lbm_synchronize(h);
                if (rc == LBM_ERR_DIVERGED) diverged = true;
                else if (rc) return rc;
            }
        }
        auto t1 = clk::now();
        t_ver += ms(tv, t1);
        t_check += ms(tn, tv);
        if (physical && !diverged) {
            rc = lbm_internal_read_fast(h, s->ver, c1);
            if (rc == LBM_ERR_DIVERGED) diverged = true;
            else if (rc) return rc;
            if (!diverged) {
                dm = std::fabs(c1[0] / c0[0] - 1.0);
                de = std::fabs(c1[4] / c0[4] - 1.0);
                // the LB's local verdict on the prediction: the largest change
                // of a node's density and temperature over the verification
                // steps, relative to the field's largest value
                unsigned long long chg[4];
                SCK(launch_field_change(s->ver, s->pred, P, s->d_chg, s->stream));
                SCK(cudaMemcpyAsync(chg, s->d_chg, sizeof chg, cudaMemcpyDeviceToHost, s->stream));
                SCK(cudaStreamSynchronize(s->stream));
                double v[4];
                std::memcpy(v, chg, sizeof v);
                dr = v[0] / std::max(v[1], 1e-300);
                dT = v[2] / std::max(v[3], 1e-300);
            }
            const auto t2 = clk::now();
            t_check += ms(t1, t2);
            t1 = t2;
            // mean interface displacement: the area that changed phase over the interface length
            const double len = 0.25 * 3.14159265358979323846 * (double)std::max(n0[2], 1ULL);
            da = (double)n1[3] / len;
        }
        n_div += diverged ? 1.0 : 0.0;
        const bool bad = !physical || diverged || !(dm <= drift_tol) || !(de <= drift_tol) || !(da <= iface_tol) ||
                         !(dr <= field_tol) || !(dT <= field_tol);
        all_dr = std::isfinite(dr) ? std::max(all_dr, dr) : INFINITY;
        all_dT = std::isfinite(dT) ? std::max(all_dT, dT) : INFINITY;
        all_dm = std::max(all_dm, dm);
        all_de = std::max(all_de, de);
        all_da = std::max(all_da, da);
        n_bad += physical ? 0.0 : 1.0;
        if (bad) {
            if (physical) {
                rc = lbm_internal_restore(h, s->snapshot);
                if (rc) return rc;
            }
            // the snapshot's step count goes with its populations
            rc = lbm_internal_set_steps(h, steps0);
            if (rc) return rc;
            auto t2 = std::chrono::steady_clock::now();
            rc = lbm_step(h, s->cfg.K + verify_steps);
            if (rc) return rc;
            rc = lbm_synchronize(h);
            if (rc) return rc;
            t_lb += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t2).count();
            fb += 1;
            have_state = false;
        } else {
            // the jump and its verification advanced the lattice by K + verify_steps
            rc = lbm_internal_set_steps(h, steps0 + s->cfg.K + verify_steps);
            if (rc) return rc;
            acc += 1;
            max_dm = std::max(max_dm, dm);
            max_de = std::max(max_de, de);
            std::memcpy(c0, c1, sizeof c0);
            std::swap(s->fields, s->ver);
            have_state = true;
        }
    }
    t_sur = t_net + t_check + t_ver;
    if (stats) {
        stats[0] = acc; stats[1] = fb; stats[2] = t_sur; stats[3] = t_lb; stats[4] = max_dm; stats[5] = max_de;
        stats[6] = all_dm; stats[7] = all_de; stats[8] = all_da; stats[9] = n_bad;
        stats[10] = n_div; stats[11] = t_prep; stats[12] = t_net; stats[13] = t_check; stats[14] = t_ver;
        stats[15] = all_dr; stats[16] = all_dT;
    }
    return LBM_OK;
}

int lbm_surrogate_destroy(lbm_surrogate* s) {
    if (!s) return LBM_OK;
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (Layer& L : s->layers) {
        s_free(L.w); s_free(L.b); s_free(L.gw); s_free(L.gb); s_free(L.mw); s_free(L.vw); s_free(L.mb);
        s_free(L.vb); s_free(L.w16); s_free(L.wflip);
    }
    release_acts(s);
    s_free(s->d_loss); s_free(s->d_cnt); s_free(s->d_status); s_free(s->d_msum); s_free(s->d_mpart); s_free(s->d_lpart); s_free(s->gpart); s_free(s->fields); s_free(s->pred); s_free(s->ver); s_free(s->d_chg); s_free(s->snapshot);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return LBM_OK;
}

}  // extern "C"
