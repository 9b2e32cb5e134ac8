// Launchers of the surrogate's BF16 tensor-core kernels (lbm_conv.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace lbm {

// x_norm = (x - off) * inv_scale per field (rho, u_x, u_y, T)
struct NormConsts {
    double off[4];
    double scale[4];
    double inv_scale[4];
};

struct ConvArgs {
    const __nv_bfloat16* in;      // [N][H][W][cin]
    const __nv_bfloat16* w;       // [9][cout][cin]
    const float* bias;            // [cout] or null
    int N, H, W;                  // W a multiple of 16
    int in_relu;                  // apply max(0, .) to the input
    const __nv_bfloat16* mask;    // [P][cout]: zero where mask <= 0 (or null)
    const __nv_bfloat16* res16;   // [P][cout] added (or null)
    const float* res32;           // [P][res32_c] added to the first res32_c channels (or null)
    int res32_c;
    __nv_bfloat16* out16;         // [P][cout] BF16 output, or
    float* out32;                 // [P][cout] FP32 output
};

size_t conv_smem_bytes(int cin, int cout);
cudaError_t launch_conv(int cin, int cout, const ConvArgs& a, cudaStream_t s, int sms);
// The same convolution on tcgen05 MMAs with tensor-memory accumulators
// (lbm_conv_tc.cu); bit 0 of the device int *status is set if a wait for
// the tensor cores ran out of time (the output is then incomplete).
cudaError_t launch_conv_tc(int cin, int cout, const ConvArgs& a, cudaStream_t s, int sms, int* status);
// The gradient reductions write per-block partial sums to `part` and add
// them in block order (no atomics, so results are reproducible bit for
// bit); grad_scratch_floats(sms) floats serve both.
size_t grad_scratch_floats(int sms);
cudaError_t launch_wgrad(int cin, int cout, const __nv_bfloat16* in, const __nv_bfloat16* dout, int N, int H, int W,
                         int in_relu, float* dw, float* part, cudaStream_t s, int sms);
// The 64 -> 64 weight gradient on tcgen05 MMAs with tensor-memory
// accumulators (lbm_conv_tc.cu; the same partial layout and block order);
// bit 0 of *status as for launch_conv_tc.
cudaError_t launch_wgrad_tc(int cin, int cout, const __nv_bfloat16* in, const __nv_bfloat16* dout, int N, int H, int W,
                            int in_relu, float* dw, float* part, cudaStream_t s, int sms, int* status);
// dw[9][cc] += the sum over blocks 0 .. nblk - 1 (in that order) of the
// partials part[nblk][3 dy][3 dx][cc]
cudaError_t launch_wgrad_sum(const float* part, int nblk, int cc, float* dw, cudaStream_t s);
cudaError_t launch_bgrad(const __nv_bfloat16* dout, long long P, int C, float* db, float* part, cudaStream_t s);
// blocks per image of the mass layer's sums: part holds 2 MASS_BLOCKS N doubles
constexpr int MASS_BLOCKS = 256;
// loss partials: part holds MSE_BLOCKS doubles
constexpr int MSE_BLOCKS = 1024;
// csum (may be null): per-image sums of (x_rho - target_rho) of the
// mass-conserving output layer, HW pixels per image
cudaError_t launch_mse(const float* out, const float* target, long long P, __nv_bfloat16* dout, double* loss,
                       const double* csum, long long HW, double* part, cudaStream_t s);
// Mass-conserving output layer on y [N*HW][16] given the input x [N*HW][4]:
// y_rho -= mean over each image of (y_rho - x_rho). With a target t, also
// sums[N + n] = sum over image n of (x_rho - t_rho) for launch_mse.
// sums: 2 N doubles of scratch.
cudaError_t launch_mass_layer(float* y, const float* x, const float* t, int N, long long HW, double* sums,
                              double* part, cudaStream_t s);
cudaError_t launch_adam(float* w, float* m, float* v, const float* g, int n, float lr, float b1, float b2, float eps,
                        float c1, float c2, cudaStream_t s);
cudaError_t launch_refresh(const float* w, int cin, int cout, int cin_real, int cout_real, __nv_bfloat16* w16,
                           __nv_bfloat16* wflip, cudaStream_t s);
cudaError_t launch_pack(const double* rho, const double* ux, const double* uy, const double* T, long long P,
                        const NormConsts& nc, __nv_bfloat16* x16, float* x32, cudaStream_t s);
cudaError_t launch_unpack(const float* y, long long P, const NormConsts& nc, double* rho, double* ux, double* uy,
                          double* T, cudaStream_t s);

// cnt[4]: liquid nodes (rho > mid), unphysical nodes, liquid-vapour edges
// of the periodic W-wide image f [4][P], and nodes whose phase differs from
// that in prev (a field set of the same shape, or null)
cudaError_t launch_field_check(const double* f, const double* prev, long long P, int W, double mid,
                               unsigned long long* cnt, cudaStream_t s);
// out[0..3] (bit patterns of doubles): max |a - b| and max |b| over the
// density plane, then the same over the temperature plane of [4][P] field sets
cudaError_t launch_field_change(const double* a, const double* b, long long P, unsigned long long* out,
                                cudaStream_t s);

}  // namespace lbm
