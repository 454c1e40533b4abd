// Network kernels of the MgNet preconditioner (FP32 on CUDA cores).
//
// One gather convolution kernel serves every convolution of the V-cycle and
// its backward pass.  A convolution is given as a tap table: for output
// pixel (gy, gx) of a "class grid" and tap t, the input pixel is
// (S gy + dy_t, S gx + dx_t) and the weight is w[(o so + i si) KK + wi_t].
//   3x3 stride 1 / stride 2 / 1x1 convolutions: one class grid = the output.
//   Transposed 4x4 stride 2 (prolongation) and the backward data of the
//   stride-2 restriction: four parity classes, each a small convolution on the
//   coarse grid whose results land at (2 gy + py, 2 gx + px).
//   Backward data of a convolution: flipped taps and swapped weight strides.
// The epilogue fuses what the V-cycle applies to a convolution result:
//   v = acc (+ bias[o]) (+ cst); raw = v; v *= gate; v *= mask > 0;
//   v = sign v (+ base) (+ y);  y = v.
// Weight gradients use the same tap tables (k_wgrad).
#include <cmath>

#include "nn_internal.h"

namespace rte {
namespace nn {
namespace {

constexpr int kTileG = 8;        // 8 x 8 class-grid pixels per CTA
constexpr int kChunk = 8;        // input channels staged per pass
constexpr int kMaxPatch = 20;    // staged patch side of the weight-gradient tile
constexpr int kSmallGrid = 4096; // class grids up to this many pixels use k_conv_small

// CTA tile: TCO output channels x (TW x TH) class-grid pixels, TCO * TW * TH =
// 4096 outputs; each of the 256 threads computes 4 channels x 4 pixels of a
// row.  TCO follows the layer's output width (16, 32 or 64) so that narrow
// layers do not idle most of the tile.
template <int TCO, int TW, int TH>
__global__ void __launch_bounds__(256) k_conv(ConvArgs a) {
    constexpr int PYM = (TH - 1) * 2 + 4, PXM = (TW - 1) * 2 + 4;   // largest staged patch
    __shared__ float xs[kChunk][PYM][PXM + 1];
    __shared__ __align__(16) float ws[kChunk][kMaxTaps][TCO];
    const int tid = threadIdx.x;
    const int tilesx = (a.Wg + TW - 1) / TW;
    const int gy0 = (blockIdx.x / tilesx) * TH, gx0 = (blockIdx.x % tilesx) * TW;
    const int co0 = blockIdx.y * TCO;
    const int b = blockIdx.z;
    const int PY = (TH - 1) * a.S + (a.tp.dymax - a.tp.dymin) + 1;
    const int PX = (TW - 1) * a.S + (a.tp.dxmax - a.tp.dxmin) + 1;
    constexpr int GROUPS = TW * TH / 4;          // pixel groups of 4 along a row
    const int tco = tid / GROUPS, tpx = tid % GROUPS;
    const int r = tpx / (TW / 4), c0 = (tpx % (TW / 4)) * 4;
    float acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[p][j] = 0.f;
    const float* xb = a.x + (size_t)b * a.Ci * a.Hi * a.Wi;
    for (int ci0 = 0; ci0 < a.Ci; ci0 += kChunk) {
        for (int e = tid; e < kChunk * PY * PX; e += 256) {
            const int ci = e / (PY * PX), rem = e - ci * PY * PX;
            const int yy = rem / PX, xx = rem - yy * PX;
            const int iy = a.S * gy0 + a.tp.dymin + yy, ix = a.S * gx0 + a.tp.dxmin + xx;
            float v = 0.f;
            if (ci0 + ci < a.Ci && iy >= 0 && iy < a.Hi && ix >= 0 && ix < a.Wi) {
                v = xb[((size_t)(ci0 + ci) * a.Hi + iy) * a.Wi + ix];
                if (a.relu_in) v = fmaxf(v, 0.f);
            }
            xs[ci][yy][xx] = v;
        }
        for (int e = tid; e < kChunk * a.tp.T * TCO; e += 256) {
            const int ci = e / (a.tp.T * TCO), rem = e - ci * a.tp.T * TCO;
            const int t = rem / TCO, co = rem - t * TCO;
            float v = 0.f;
            if (ci0 + ci < a.Ci && co0 + co < a.Co)
                v = a.w[((size_t)(co0 + co) * a.so + (size_t)(ci0 + ci) * a.si) * a.KK + a.tp.wi[t]];
            ws[ci][t][co] = v;
        }
        __syncthreads();
        const int nci = min(kChunk, a.Ci - ci0);
        for (int ci = 0; ci < nci; ++ci) {
            for (int t = 0; t < a.tp.T; ++t) {
                const int yy = a.S * r + a.tp.dy[t] - a.tp.dymin;
                const int xx0 = a.S * c0 + a.tp.dx[t] - a.tp.dxmin;
                float xv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) xv[j] = xs[ci][yy][xx0 + a.S * j];
                const float4 wv = *reinterpret_cast<const float4*>(&ws[ci][t][tco * 4]);
                const float wa[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[p][j] = fmaf(wa[p], xv[j], acc[p][j]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int co = co0 + tco * 4 + p;
        if (co >= a.Co) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gy = gy0 + r, gx = gx0 + c0 + j;
            if (gy >= a.Hg || gx >= a.Wg) continue;
            const int oy = a.OS * gy + a.OY0, ox = a.OS * gx + a.OX0;
            const size_t idx = (((size_t)b * a.Co + co) * a.Ho + oy) * a.Wo + ox;
            float v = acc[p][j];
            if (a.bias) v += a.bias[co];
            v += a.cst;
            if (a.raw) a.raw[idx] = v;
            if (a.gate)
                v *= a.gate[a.gate_bcast ? (((size_t)co * a.Ho + oy) * a.Wo + ox) : idx];
            if (a.mask && !(a.mask[idx] > 0.f)) v = 0.f;
            v *= a.sign;
            if (a.base) v += a.base[idx];
            if (a.accumulate) v += a.y[idx];
            a.y[idx] = v;
        }
    }
}

// Small class grids (coarse V-cycle levels): one output per thread, so even an
// 8 x 8 grid with 64 channels spreads over 16 CTAs instead of one.  Threads of
// a warp share the output channel (weights broadcast) and cover consecutive
// pixels (coalesced inputs, reused through L1 by the neighbouring taps).
__global__ void __launch_bounds__(256) k_conv_small(ConvArgs a) {
    const int64_t total = (int64_t)a.B * a.Co * a.Hg * a.Wg;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int gx = (int)(e % a.Wg);
    const int gy = (int)((e / a.Wg) % a.Hg);
    const int co = (int)((e / ((int64_t)a.Wg * a.Hg)) % a.Co);
    const int b = (int)(e / ((int64_t)a.Wg * a.Hg * a.Co));
    const float* xb = a.x + (size_t)b * a.Ci * a.Hi * a.Wi;
    float acc = 0.f;
    for (int t = 0; t < a.tp.T; ++t) {
        const int iy = a.S * gy + a.tp.dy[t], ix = a.S * gx + a.tp.dx[t];
        if (iy < 0 || iy >= a.Hi || ix < 0 || ix >= a.Wi) continue;
        const float* xp = xb + (size_t)iy * a.Wi + ix;
        const float* wp = a.w + (size_t)co * a.so * a.KK + a.tp.wi[t];
        const size_t xs = (size_t)a.Hi * a.Wi, wstep = (size_t)a.si * a.KK;
        if (a.relu_in) {
            for (int ci = 0; ci < a.Ci; ++ci) acc = fmaf(__ldg(wp + ci * wstep), fmaxf(__ldg(xp + ci * xs), 0.f), acc);
        } else {
            for (int ci = 0; ci < a.Ci; ++ci) acc = fmaf(__ldg(wp + ci * wstep), __ldg(xp + ci * xs), acc);
        }
    }
    const int oy = a.OS * gy + a.OY0, ox = a.OS * gx + a.OX0;
    const size_t idx = (((size_t)b * a.Co + co) * a.Ho + oy) * a.Wo + ox;
    float v = acc;
    if (a.bias) v += a.bias[co];
    v += a.cst;
    if (a.raw) a.raw[idx] = v;
    if (a.gate) v *= a.gate[a.gate_bcast ? (((size_t)co * a.Ho + oy) * a.Wo + ox) : idx];
    if (a.mask && !(a.mask[idx] > 0.f)) v = 0.f;
    v *= a.sign;
    if (a.base) v += a.base[idx];
    if (a.accumulate) v += a.y[idx];
    a.y[idx] = v;
}

// dW[(o so + i si) KK + wi_t] += sum_{b, gy, gx} G[b][o][OS gy + OY0][OS gx + OX0]
//                                      * X[b][i][S gy + dy_t][S gx + dx_t]
// Deterministic in two launches.  k_wgrad: CTA (x, y) owns 16 o x 16 i
// (y) and the work items q = x, x + P, x + 2P, ... of the (batch entry,
// 8 x 8 class-grid tile) list; it accumulates them in that order in
// registers (one sum per tap) and writes its partial sums to
// part[x][o][i][t].  k_wgrad_reduce adds the P partials of every weight in
// order x = 0..P-1 onto dW.  No atomics: a training step gives the same bits
// on every run.
__global__ void __launch_bounds__(256) k_wgrad(WgradArgs a, int P, float* __restrict__ part) {
    __shared__ float gs[16][kTileG * kTileG];
    __shared__ float xs[16][kMaxPatch][kMaxPatch + 1];
    const int tid = threadIdx.x;
    const int tilesx = (a.Wg + kTileG - 1) / kTileG;
    const int tiles = tilesx * ((a.Hg + kTileG - 1) / kTileG);
    const int items = tiles * a.B;
    const int otiles = (a.Co + 15) / 16;
    const int o0 = (blockIdx.y % otiles) * 16, i0 = (blockIdx.y / otiles) * 16;
    const int PY = (kTileG - 1) * a.S + (a.tp.dymax - a.tp.dymin) + 1;
    const int PX = (kTileG - 1) * a.S + (a.tp.dxmax - a.tp.dxmin) + 1;
    const int o = tid >> 4, i = tid & 15;
    const bool own = (o0 + o < a.Co) && (i0 + i < a.Ci);
    float acc[kMaxTaps];
#pragma unroll
    for (int t = 0; t < kMaxTaps; ++t) acc[t] = 0.f;
    for (int q = blockIdx.x; q < items; q += P) {
        const int b = q / tiles, tile = q - b * tiles;
        const int gy0 = (tile / tilesx) * kTileG, gx0 = (tile % tilesx) * kTileG;
        __syncthreads();                 // the previous item's reads are done
        for (int e = tid; e < 16 * kTileG * kTileG; e += 256) {
            const int oo = e / (kTileG * kTileG), p = e - oo * kTileG * kTileG;
            const int gy = gy0 + p / kTileG, gx = gx0 + p % kTileG;
            float v = 0.f;
            if (o0 + oo < a.Co && gy < a.Hg && gx < a.Wg)
                v = a.g[(((size_t)b * a.Co + o0 + oo) * a.Hgo + a.OS * gy + a.OY0) * a.Wgo + a.OS * gx + a.OX0];
            gs[oo][p] = v;
        }
        for (int e = tid; e < 16 * PY * PX; e += 256) {
            const int ii = e / (PY * PX), rem = e - ii * PY * PX;
            const int yy = rem / PX, xx = rem - yy * PX;
            const int iy = a.S * gy0 + a.tp.dymin + yy, ix = a.S * gx0 + a.tp.dxmin + xx;
            float v = 0.f;
            if (i0 + ii < a.Ci && iy >= 0 && iy < a.Hi && ix >= 0 && ix < a.Wi) {
                v = a.x[(((size_t)b * a.Ci + i0 + ii) * a.Hi + iy) * a.Wi + ix];
                if (a.relu_in) v = fmaxf(v, 0.f);
            }
            xs[ii][yy][xx] = v;
        }
        __syncthreads();
        if (own) {
#pragma unroll
            for (int t = 0; t < kMaxTaps; ++t) {
                if (t < a.tp.T) {
                    const int ty = a.tp.dy[t] - a.tp.dymin, tx = a.tp.dx[t] - a.tp.dxmin;
                    float s = 0.f;          // the tile's sum, then added (two-level summation)
                    for (int p = 0; p < kTileG * kTileG; ++p) {
                        const int py = p / kTileG, px = p - py * kTileG;
                        s = fmaf(gs[o][p], xs[i][a.S * py + ty][a.S * px + tx], s);
                    }
                    acc[t] += s;
                }
            }
        }
    }
    if (!own) return;
    float* dst = part + (((size_t)blockIdx.x * a.Co + o0 + o) * a.Ci + i0 + i) * a.tp.T;
#pragma unroll
    for (int t = 0; t < kMaxTaps; ++t)
        if (t < a.tp.T) dst[t] = acc[t];
}

// dW[(o so + i si) KK + wi_t] += sum_{x < P} part[x][o][i][t], x ascending.
// The taps of one launch address distinct weights (checked on the host), so
// every weight has one writer.
__global__ void k_wgrad_reduce(WgradArgs a, int P, const float* __restrict__ part) {
    const size_t per = (size_t)a.Co * a.Ci * a.tp.T;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < per; e += (size_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int x = 0; x < P; ++x) s += part[(size_t)x * per + e];
        const int t = (int)(e % a.tp.T);
        const size_t oi = e / a.tp.T;
        const int i = (int)(oi % a.Ci), o = (int)(oi / a.Ci);
        a.dw[((size_t)o * a.so + (size_t)i * a.si) * a.KK + a.tp.wi[t]] += s;
    }
}

// Per-channel statistics over (B, H, W): mean and 1/sqrt(var + eps) (biased
// variance, two passes in FP64).
__global__ void k_bn_stats(const float* __restrict__ x, int B, int C, int HW, float eps,
                           float* __restrict__ mean, float* __restrict__ invstd) {
    __shared__ double red[32];
    const int c = blockIdx.x;
    double s = 0.0;
    for (int e = threadIdx.x; e < B * HW; e += blockDim.x) {
        const int b = e / HW, p = e - b * HW;
        s += x[((size_t)b * C + c) * HW + p];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        red[0] = t / ((double)B * HW);
    }
    __syncthreads();
    const double mu = red[0];
    __syncthreads();
    double v = 0.0;
    for (int e = threadIdx.x; e < B * HW; e += blockDim.x) {
        const int b = e / HW, p = e - b * HW;
        const double d = x[((size_t)b * C + c) * HW + p] - mu;
        v += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        mean[c] = (float)mu;
        invstd[c] = (float)(1.0 / sqrt(t / ((double)B * HW) + (double)eps));
    }
}

// y = ReLU(gamma (x - mean) invstd + beta)
__global__ void k_bn_relu(const float* __restrict__ x, int B, int C, int HW,
                          const float* __restrict__ mean, const float* __restrict__ invstd,
                          const float* __restrict__ gamma, const float* __restrict__ beta,
                          float* __restrict__ y) {
    const size_t n = (size_t)B * C * HW;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)((e / HW) % C);
        const float v = gamma[c] * (x[e] - mean[c]) * invstd[c] + beta[c];
        y[e] = fmaxf(v, 0.f);
    }
}

// Backward of y = ReLU(BN(x)): per channel sums S1 = sum g', S2 = sum g' xh
// with g' = g [y > 0]; dgamma += S2, dbeta += S1; then
// dx = gamma invstd / cnt (cnt g' - S1 - xh S2).
__global__ void k_bn_relu_bwd(const float* __restrict__ x, const float* __restrict__ y,
                              const float* __restrict__ g, int B, int C, int HW,
                              const float* __restrict__ mean, const float* __restrict__ invstd,
                              const float* __restrict__ gamma, float* __restrict__ dgamma,
                              float* __restrict__ dbeta, float* __restrict__ dx) {
    __shared__ double r1[32], r2[32];
    const int c = blockIdx.x;
    const float mu = mean[c], is = invstd[c];
    double s1 = 0.0, s2 = 0.0;
    for (int e = threadIdx.x; e < B * HW; e += blockDim.x) {
        const int b = e / HW, p = e - b * HW;
        const size_t idx = ((size_t)b * C + c) * HW + p;
        const float gp = y[idx] > 0.f ? g[idx] : 0.f;
        const float xh = (x[idx] - mu) * is;
        s1 += gp;
        s2 += (double)gp * xh;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) { r1[threadIdx.x >> 5] = s1; r2[threadIdx.x >> 5] = s2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t1 += r1[w]; t2 += r2[w]; }
        r1[0] = t1;
        r2[0] = t2;
        dgamma[c] += (float)t2;
        dbeta[c] += (float)t1;
    }
    __syncthreads();
    const double S1 = r1[0], S2 = r2[0];
    const double cnt = (double)B * HW;
    for (int e = threadIdx.x; e < B * HW; e += blockDim.x) {
        const int b = e / HW, p = e - b * HW;
        const size_t idx = ((size_t)b * C + c) * HW + p;
        const float gp = y[idx] > 0.f ? g[idx] : 0.f;
        const double xh = ((double)x[idx] - mu) * is;
        dx[idx] = (float)((double)gamma[c] * is / cnt * (cnt * gp - S1 - xh * S2));
    }
}

// backward of v = sign raw * gate with one gate shared by B samples:
// out[b] = sign g[b] gate ; dgate += sum_b sign g[b] raw[b]
__global__ void k_gate_bwd(const float* __restrict__ g, const float* __restrict__ gate,
                           const float* __restrict__ raw, float sign, int B, size_t chw,
                           float* __restrict__ out, float* __restrict__ dgate) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < chw; e += (size_t)gridDim.x * blockDim.x) {
        const float ge = gate[e];
        float acc = 0.f;
        for (int b = 0; b < B; ++b) {
            const float gv = sign * g[(size_t)b * chw + e];
            out[(size_t)b * chw + e] = gv * ge;
            acc = fmaf(gv, raw[(size_t)b * chw + e], acc);
        }
        dgate[e] += acc;
    }
}

__global__ void k_scale_copy(float* __restrict__ y, const float* __restrict__ x, float alpha, size_t n) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        y[e] = alpha * x[e];
}

__global__ void k_axpy_f(float* __restrict__ y, const float* __restrict__ x, float alpha, size_t n) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        y[e] += alpha * x[e];
}

// per-channel sum over (B, H, W) into out[c] (+=): gradient of a head bias
__global__ void k_channel_sum(const float* __restrict__ g, int B, int C, int HW, float* __restrict__ out) {
    __shared__ float red[32];
    const int c = blockIdx.x;
    float s = 0.f;
    for (int e = threadIdx.x; e < B * HW; e += blockDim.x) {
        const int b = e / HW, p = e - b * HW;
        s += g[((size_t)b * C + c) * HW + p];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        out[c] += t;
    }
}

// Adam (Kingma & Ba): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
// p -= lr (m / c1) / (sqrt(v / c2) + eps), c_i = 1 - b_i^t.  The constants
// 1 - b_i and c_i come from the host, computed in FP64 and rounded once (in
// FP32, 1 - 0.999f is 1.3e-5 away from 1e-3).
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, size_t n, float lr, float b1, float b2, float omb1,
                       float omb2, float eps, float c1, float c2) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[e];
        const float mi = b1 * m[e] + omb1 * gi;
        const float vi = b2 * v[e] + omb2 * gi * gi;
        m[e] = mi;
        v[e] = vi;
        p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

int ew_blocks(size_t n) {
    size_t b = (n + 255) / 256;
    return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

thread_local Counters* tl_counters = nullptr;

void conv(const ConvArgs& a, cudaStream_t st) {
    if (a.tp.T > kMaxTaps) throw StatusError{RTE_EINVAL, "too many taps"};
    if (a.S < 1 || a.S > 2 || a.tp.dymax - a.tp.dymin > 3 || a.tp.dxmax - a.tp.dxmin > 3)
        throw StatusError{RTE_EINVAL, "convolution stride or tap span too large"};
    if (tl_counters) {
        tl_counters->launches += 1;
        tl_counters->flops += 2.0 * a.B * a.Co * (double)a.Hg * a.Wg * a.Ci * a.tp.T;
    }
    auto launch = [&](auto kern, int tco, int tw, int th) {
        const int tiles = ((a.Hg + th - 1) / th) * ((a.Wg + tw - 1) / tw);
        dim3 grid(tiles, (a.Co + tco - 1) / tco, a.B);
        kern<<<grid, 256, 0, st>>>(a);
    };
    if ((int64_t)a.Hg * a.Wg <= kSmallGrid) {
        const int64_t total = (int64_t)a.B * a.Co * a.Hg * a.Wg;
        k_conv_small<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(a);
    } else if (a.Co <= 16)
        launch(k_conv<16, 16, 16>, 16, 16, 16);
    else if (a.Co <= 32)
        launch(k_conv<32, 16, 8>, 32, 16, 8);
    else
        launch(k_conv<64, 8, 8>, 64, 8, 8);
    check(cudaGetLastError(), "k_conv");
}

thread_local WgradScratch* tl_wgrad_scratch = nullptr;

void wgrad(const WgradArgs& a, cudaStream_t st) {
    const int PY = (kTileG - 1) * a.S + (a.tp.dymax - a.tp.dymin) + 1;
    const int PX = (kTileG - 1) * a.S + (a.tp.dxmax - a.tp.dxmin) + 1;
    if (PY > kMaxPatch || PX > kMaxPatch || a.tp.T > kMaxTaps || a.tp.T < 1)
        throw StatusError{RTE_EINVAL, "wgrad tile too large"};
    for (int t = 0; t < a.tp.T; ++t)
        for (int u = 0; u < t; ++u)
            if (a.tp.wi[t] == a.tp.wi[u]) throw StatusError{RTE_EINVAL, "wgrad: repeated weight tap"};
    const WgradScratch* ws = tl_wgrad_scratch;
    if (!ws || !ws->part) throw StatusError{RTE_EINVAL, "wgrad: no partial-sum scratch"};
    const int tiles = ((a.Hg + kTileG - 1) / kTileG) * ((a.Wg + kTileG - 1) / kTileG);
    const int items = tiles * a.B;
    const int oi = ((a.Co + 15) / 16) * ((a.Ci + 15) / 16);
    const size_t per = (size_t)a.Co * a.Ci * a.tp.T;
    // about four CTAs per SM in all, at most one partial block per work item,
    // and the partials within the scratch
    int P = (4 * ws->num_sms + oi - 1) / oi;
    if (P > items) P = items;
    const size_t fit = ws->cap / per;
    if (fit < 1) throw StatusError{RTE_EINVAL, "wgrad: layer larger than the partial-sum scratch"};
    if ((size_t)P > fit) P = (int)fit;
    if (P < 1) P = 1;
    dim3 grid(P, oi);
    k_wgrad<<<grid, 256, 0, st>>>(a, P, ws->part);
    const size_t rb = (per + 255) / 256;
    k_wgrad_reduce<<<(unsigned)(rb < 4096 ? rb : 4096), 256, 0, st>>>(a, P, ws->part);
    check(cudaGetLastError(), "k_wgrad");
}

void bn_stats(const float* x, int B, int C, int HW, float* mean, float* invstd, cudaStream_t st) {
    k_bn_stats<<<C, 256, 0, st>>>(x, B, C, HW, 1e-5f, mean, invstd);
    check(cudaGetLastError(), "k_bn_stats");
}

void bn_relu(const float* x, int B, int C, int HW, const float* mean, const float* invstd,
             const float* gamma, const float* beta, float* y, cudaStream_t st) {
    const size_t n = (size_t)B * C * HW;
    k_bn_relu<<<ew_blocks(n), 256, 0, st>>>(x, B, C, HW, mean, invstd, gamma, beta, y);
    check(cudaGetLastError(), "k_bn_relu");
}

void bn_relu_bwd(const float* x, const float* y, const float* g, int B, int C, int HW,
                 const float* mean, const float* invstd, const float* gamma, float* dgamma,
                 float* dbeta, float* dx, cudaStream_t st) {
    k_bn_relu_bwd<<<C, 256, 0, st>>>(x, y, g, B, C, HW, mean, invstd, gamma, dgamma, dbeta, dx);
    check(cudaGetLastError(), "k_bn_relu_bwd");
}

void gate_bwd(const float* g, const float* gate, const float* raw, float sign, int B, size_t chw,
              float* out, float* dgate, cudaStream_t st) {
    k_gate_bwd<<<ew_blocks(chw), 256, 0, st>>>(g, gate, raw, sign, B, chw, out, dgate);
    check(cudaGetLastError(), "k_gate_bwd");
}

void scale_copy(float* y, const float* x, float alpha, size_t n, cudaStream_t st) {
    k_scale_copy<<<ew_blocks(n), 256, 0, st>>>(y, x, alpha, n);
    check(cudaGetLastError(), "k_scale_copy");
}

void axpy(float* y, const float* x, float alpha, size_t n, cudaStream_t st) {
    k_axpy_f<<<ew_blocks(n), 256, 0, st>>>(y, x, alpha, n);
    check(cudaGetLastError(), "k_axpy_f");
}

void channel_sum(const float* g, int B, int C, int HW, float* out, cudaStream_t st) {
    k_channel_sum<<<C, 256, 0, st>>>(g, B, C, HW, out);
    check(cudaGetLastError(), "k_channel_sum");
}

void adam(float* p, const float* g, float* m, float* v, size_t n, float lr, int step, cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f;
    // bias corrections 1 - beta^t in FP64, then rounded once: in FP32,
    // 1 - 0.999f^t loses about five digits to cancellation at small t
    const float c1 = (float)(1.0 - std::pow(0.9, (double)step));
    const float c2 = (float)(1.0 - std::pow(0.999, (double)step));
    k_adam<<<ew_blocks(n), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, (float)(1.0 - 0.9), (float)(1.0 - 0.999),
                                         1e-8f, c1, c2);
    check(cudaGetLastError(), "k_adam");
}

// ---------------------------------------------------------------- tap tables
Taps taps_conv(int k, int pad) {
    Taps t{};
    t.T = k * k;
    for (int ky = 0; ky < k; ++ky)
        for (int kx = 0; kx < k; ++kx) {
            const int q = ky * k + kx;
            t.dy[q] = ky - pad;
            t.dx[q] = kx - pad;
            t.wi[q] = q;
        }
    t.finish();
    return t;
}

Taps taps_conv_flipped(int k, int pad) {
    Taps t{};
    t.T = k * k;
    for (int ky = 0; ky < k; ++ky)
        for (int kx = 0; kx < k; ++kx) {
            const int q = ky * k + kx;
            t.dy[q] = pad - ky;
            t.dx[q] = pad - kx;
            t.wi[q] = q;
        }
    t.finish();
    return t;
}

// Scatter of a stride-2 kernel of size k (pad 1) onto fine-grid parity
// class (py, px): fine pixel 2 gy + py receives coarse pixel gy + d from
// kernel row ky when 2 (gy + d) + ky - 1 = 2 gy + py, i.e. ky = py + 1 - 2 d.
Taps taps_parity(int k, int py, int px) {
    Taps t{};
    t.T = 0;
    for (int ky = 0; ky < k; ++ky) {
        if (((py + 1 - ky) & 1) != 0) continue;
        const int dy = (py + 1 - ky) / 2;
        for (int kx = 0; kx < k; ++kx) {
            if (((px + 1 - kx) & 1) != 0) continue;
            const int dx = (px + 1 - kx) / 2;
            t.dy[t.T] = dy;
            t.dx[t.T] = dx;
            t.wi[t.T] = ky * k + kx;
            ++t.T;
        }
    }
    t.finish();
    return t;
}

}  // namespace nn
}  // namespace rte
