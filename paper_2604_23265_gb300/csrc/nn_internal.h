// Internal interface of the network kernels (nn_kernels.cu).
#pragma once

#include <cuda.h>

#include "rte_internal.h"

namespace rte {
namespace nn {

constexpr int kMaxTaps = 16;
constexpr int kTcMaxBatch = 16;     // samples of one batched tensor-core launch

// Taps of a gather convolution: input pixel (S gy + dy[t], S gx + dx[t]),
// weight offset wi[t] inside the kernel window.
struct Taps {
    int T = 0;
    int dy[kMaxTaps] = {};
    int dx[kMaxTaps] = {};
    int wi[kMaxTaps] = {};
    int dymin = 0, dymax = 0, dxmin = 0, dxmax = 0;
    void finish() {
        dymin = dxmin = 1 << 20;
        dymax = dxmax = -(1 << 20);
        for (int t = 0; t < T; ++t) {
            dymin = dy[t] < dymin ? dy[t] : dymin;
            dymax = dy[t] > dymax ? dy[t] : dymax;
            dxmin = dx[t] < dxmin ? dx[t] : dxmin;
            dxmax = dx[t] > dxmax ? dx[t] : dxmax;
        }
    }
};

struct ConvArgs {
    const float* x = nullptr;        // [B][Ci][Hi][Wi]
    int B = 1, Ci = 0, Hi = 0, Wi = 0;
    const float* w = nullptr;        // w[(o so + i si) KK + wi]
    int so = 0, si = 0, KK = 1;
    int Co = 0;
    int Hg = 0, Wg = 0, S = 1;       // class grid and input stride
    int OS = 1, OY0 = 0, OX0 = 0;    // output placement
    float* y = nullptr;              // [B][Co][Ho][Wo]
    int Ho = 0, Wo = 0;
    const float* bias = nullptr;     // per output channel
    float cst = 0.f;
    float* raw = nullptr;            // stores acc (+bias +cst) before gating
    const float* gate = nullptr;     // [B][Co][Ho][Wo], or [Co][Ho][Wo] if gate_bcast
    int gate_bcast = 0;
    const float* mask = nullptr;     // keep where mask > 0
    float sign = 1.f;
    const float* base = nullptr;     // added after sign
    int accumulate = 0;              // y += ...
    int relu_in = 0;                 // ReLU applied to x on load
    Taps tp;
};

struct WgradArgs {
    const float* g = nullptr;        // [B][Co][Hgo][Wgo] (gradient of the output)
    int B = 1, Co = 0, Hgo = 0, Wgo = 0;
    int Hg = 0, Wg = 0, OS = 1, OY0 = 0, OX0 = 0;
    const float* x = nullptr;        // [B][Ci][Hi][Wi]
    int Ci = 0, Hi = 0, Wi = 0, S = 1;
    int relu_in = 0;
    float* dw = nullptr;             // accumulated: dw[(o so + i si) KK + wi]
    int so = 0, si = 0, KK = 1;
    Taps tp;
};

// counters of the calling network (launches and FP32 flops), may be null
struct Counters {
    long long launches = 0;
    double flops = 0.0;
};
extern thread_local Counters* tl_counters;

// Partial-sum scratch of the deterministic weight gradient (wgrad): cap floats
// on the device; set by the network around its backward pass.
struct WgradScratch {
    float* part = nullptr;
    size_t cap = 0;
    int num_sms = 1;
};
extern thread_local WgradScratch* tl_wgrad_scratch;

void conv(const ConvArgs& a, cudaStream_t st);
// Tensor-core (tcgen05) gather convolution of the inference forward pass
// (conv_tc.cu): BF16 operands, FP32 accumulation.  Activations are BF16 in the
// channel-chunked layout C8 = [B][ceil(C/8)][H][W][8] (16-byte aligned);
// weights are packed by tc_pack.  Output pixel (OS gy + oy0, OS gx + ox0) of
// class-grid pixel (gy, gx) of a class receives
//   v = sign (sum_t sum_i X[b][i][S gy + dy_t][S gx + dx_t] W[t][i][o]) gate[o] (+ base)
struct TcConv {
    CUtensorMap tmap;                // filled by tc_conv (TMA halo loads of x8)
    const void* x8 = nullptr;        // BF16 C8 input, or
    const double* x64 = nullptr;     // FP64 [B][Ci][Hi][Wi] input (converted on load)
    int B = 1, Ci = 0, Hi = 0, Wi = 0;
    int relu_in = 0;                 // ReLU applied to the gathered input
    const void* w = nullptr;         // packed weights (tc_pack of the classes T taps: tc_weight_bytes bytes)
    int Co = 0;
    int Hg = 0, Wg = 0, S = 1;       // class grid and input stride
    int OS = 1;                      // output placement OS g + (oy0, ox0)[class]
    int Ho = 0, Wo = 0;
    int T = 0;                       // taps per class
    int classes = 1;                 // class c uses taps c T .. c T + T - 1
    int dy[kMaxTaps] = {}, dx[kMaxTaps] = {};
    int oy0[4] = {}, ox0[4] = {};
    const float* gate = nullptr;     // FP32 [Co][Ho][Wo], shared by the batch
    float sign = 1.f;
    const void* base8 = nullptr;     // BF16 C8 of the output's shape, or
    const double* base64 = nullptr;  // FP64 [B][Co][Ho][Wo]
    void* y8 = nullptr;              // BF16 C8 output, or
    float* y32 = nullptr;            // FP32 [B][Co][Ho][Wo] output
    // per-sample pointers (batched != 0; B <= kTcMaxBatch), used instead of
    // the batch-strided pointers above: a batch of samples from different
    // solves, each with its own input, output and medium
    int batched = 0;
    const double* x64_b[kTcMaxBatch] = {};    // [Ci][Hi][Wi] each
    const float* gate_b[kTcMaxBatch] = {};    // [Co][Ho][Wo] each
    const double* base64_b[kTcMaxBatch] = {}; // [Co][Ho][Wo] each
    float* y32_b[kTcMaxBatch] = {};           // [Co][Ho][Wo] each
    // FP32 input / base per sample (batched only), in place of x64_b / base64_b
    const float* x32_b[kTcMaxBatch] = {};     // [Ci][Hi][Wi] each
    const float* base32_b[kTcMaxBatch] = {};  // [Co][Ho][Wo] each
};
// Bytes of the packed weights of T taps (classes x taps per class): the
// resident layout, or the streamed one for layers whose per-CTA weights
// exceed the resident limit or that have more than 256 output channels.
size_t tc_weight_bytes(int T, int classes, int Ci, int Co);
// packs W[t][i][o] = w[(o so + i si) KK + wi_t] into dst (tc_weight_bytes)
void tc_pack(const float* w, int so, int si, int KK, const Taps& tp, int classes, int Ci, int Co, void* dst,
             cudaStream_t st);
// pdl: programmatic dependent launch (the weights must not be written by the
// previous kernel in the stream)
void tc_conv(const TcConv& a, bool pdl, cudaStream_t st);
// 1 once a bounded wait of the tensor-core kernel expired (reset on request).
int conv_tc_status(bool reset);
// dw += the weight gradient of one convolution; deterministic (per-CTA
// partial sums in tl_wgrad_scratch, added in a fixed order, no atomics)
void wgrad(const WgradArgs& a, cudaStream_t st);
void bn_stats(const float* x, int B, int C, int HW, float* mean, float* invstd, cudaStream_t st);
void bn_relu(const float* x, int B, int C, int HW, const float* mean, const float* invstd,
             const float* gamma, const float* beta, float* y, cudaStream_t st);
void bn_relu_bwd(const float* x, const float* y, const float* g, int B, int C, int HW,
                 const float* mean, const float* invstd, const float* gamma, float* dgamma,
                 float* dbeta, float* dx, cudaStream_t st);
// out[b] = sign g[b] gate ; dgate += sum_b sign g[b] raw[b]   (gate shared by the B samples)
void gate_bwd(const float* g, const float* gate, const float* raw, float sign, int B, size_t chw,
              float* out, float* dgate, cudaStream_t st);
// y = x (+)= ...: small helpers
void scale_copy(float* y, const float* x, float alpha, size_t n, cudaStream_t st);
void axpy(float* y, const float* x, float alpha, size_t n, cudaStream_t st);
void channel_sum(const float* g, int B, int C, int HW, float* out, cudaStream_t st);
void adam(float* p, const float* g, float* m, float* v, size_t n, float lr, int step, cudaStream_t st);

Taps taps_conv(int k, int pad);
Taps taps_conv_flipped(int k, int pad);
Taps taps_parity(int k, int py, int px);

}  // namespace nn
}  // namespace rte
