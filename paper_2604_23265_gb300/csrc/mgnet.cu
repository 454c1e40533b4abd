// MgNet preconditioner (Sec. 3): CoeffNet + MgNet V-cycle, the physics-informed
// loss (Eq. loss), its gradient and Adam, all on the device.
//
// Network (readings of Sec. 3.2-3.3):
//   CoeffNet, level l: z = conv3x3(g_{l-1}, stride 1 at l = 0 else 2),
//     g_l = ReLU(BN(z)); a_l = 1 + head_a(g_l), ainv_l = 1 + head_ainv(g_l).
//   MgNet: f_0 = lift(x); smoothing u <- u + (B_l * act(f - (A_l * u) o a_l)) o ainv_l
//     with act the identity (default) or ReLU;
//     restriction f_{l+1} = R_l *_{s2} (f_l - (A_l * u_l) o a_l);
//     prolongation u_l <- u_l + P_l *^T u_{l+1}; one pre- and one
//     post-smoothing step per level, two on the coarsest;
//     psi_d = x + proj(u_0), x = r / rms(r), output rms(r) psi_d.
// The network works in face-flux space; the Krylov operator there is
// B = A D = I - P R (block-Jacobi preconditioned), so the loss of Eq. loss is
// ||x - B psi_d|| / ||x||, and its gradient uses B^T = I - R^T P.
// A batch is several right-hand sides of one medium: CoeffNet runs once and
// its batch statistics are the medium's own, exactly as at inference.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <stdexcept>
#include <string>

#include "mgnet_internal.h"
#include "nn_internal.h"

namespace rte {
namespace {
using nn::ConvArgs;
using nn::Taps;
using nn::WgradArgs;

struct Param {
    std::string name;
    size_t off = 0, count = 0;
};

struct Features {            // CoeffNet outputs of one medium for one weight version
    uint64_t version = ~0ull;
    uint64_t stamp = 0;      // last use (least recently used entries are evicted)
    int I = 0;
    void* block = nullptr;
    std::vector<float*> zc, gc, mean, inv, a, ai;
};

}  // namespace
}  // namespace rte

struct mgnet {
    int M = 0, L = 0, c0 = 0, cmax = 0, cc = 0, ccmax = 0, cin = 4;
    int act = 0;                     // smoother activation: 0 identity, 1 ReLU
    int prec = 1;                    // inference convolutions: 0 FP32 CUDA cores, 1 BF16 tensor cores
    int loss = 0;                    // training loss: 0 plain (Eq. loss), 1 ATFPS-filtered (Eq. loss_delta)
    int fault = 0;                   // host-side fault injection: 1 = every preconditioner output is NaN
    void* lscr = nullptr;            // scratch of the filtered loss
    size_t lscr_bytes = 0;
    // tensor-core inference path: BF16 C8 activations, packed weights
    void* tc_ws = nullptr;
    size_t tc_ws_bytes = 0;
    void* tcw = nullptr;
    size_t tcw_bytes = 0;
    uint64_t tcw_version = ~0ull;
    cudaStream_t stream = nullptr;
    std::string err;
    std::vector<rte::Param> params;
    std::map<std::string, size_t> off;
    size_t np = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    int step = 0;
    uint64_t version = 1;
    // activations
    int wsB = 0, wsI = 0;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    std::map<uint64_t, rte::Features> feats;   // by context uid, at most kFeatureCache entries
    uint64_t fclock = 0;
    // helpers for the per-sample scalars
    double* d_scal = nullptr;
    double* h_scal = nullptr;
    double* d_part = nullptr;        // [2 x 2048] block partial sums (inside d_scal's allocation)
    double* fin64 = nullptr;         // FP64 copy of an FP32 input (CUDA-core forward)
    size_t fin64_n = 0;

    int C(int l) const { int c = c0 << l; return c < cmax ? c : cmax; }
    int Cc(int l) const { int c = cc << l; return c < ccmax ? c : ccmax; }
};

namespace rte {
namespace {

// ------------------------------------------------------------------ params
void add_param(mgnet* n, const std::string& name, size_t count) {
    n->params.push_back({name, n->np, count});
    n->off[name] = n->np;
    n->np += count;
}

void build_params(mgnet* n) {
    const int L = n->L;
    for (int l = 0; l < L; ++l) {
        const int cin = l == 0 ? n->cin : n->Cc(l - 1);
        add_param(n, "coef" + std::to_string(l) + ".w", (size_t)n->Cc(l) * cin * 9);
        add_param(n, "coef" + std::to_string(l) + ".gamma", n->Cc(l));
        add_param(n, "coef" + std::to_string(l) + ".beta", n->Cc(l));
        add_param(n, "a" + std::to_string(l) + ".w", (size_t)n->C(l) * n->Cc(l));
        add_param(n, "a" + std::to_string(l) + ".b", n->C(l));
        add_param(n, "ainv" + std::to_string(l) + ".w", (size_t)n->C(l) * n->Cc(l));
        add_param(n, "ainv" + std::to_string(l) + ".b", n->C(l));
    }
    add_param(n, "lift.w", (size_t)n->C(0) * 2 * n->M);
    for (int l = 0; l < L; ++l) {
        add_param(n, "A" + std::to_string(l) + ".w", (size_t)n->C(l) * n->C(l) * 9);
        add_param(n, "B" + std::to_string(l) + ".w", (size_t)n->C(l) * n->C(l) * 9);
    }
    for (int l = 0; l + 1 < L; ++l) {
        add_param(n, "R" + std::to_string(l) + ".w", (size_t)n->C(l + 1) * n->C(l) * 9);
        add_param(n, "P" + std::to_string(l) + ".w", (size_t)n->C(l + 1) * n->C(l) * 16);
    }
    add_param(n, "proj.w", (size_t)2 * n->M * n->C(0));
}

float* P(mgnet* n, const std::string& name) { return n->p + n->off.at(name); }
float* G(mgnet* n, const std::string& name) { return n->g + n->off.at(name); }
std::string sl(const char* s, int l) { return std::string(s) + std::to_string(l) + ".w"; }

// ------------------------------------------------------------------ arena
struct Arena {
    char* base;
    size_t used = 0, cap;
    float* f(size_t count) {
        size_t bytes = (count * sizeof(float) + 255) & ~(size_t)255;
        if (used + bytes > cap) throw StatusError{RTE_ENOMEM, "network workspace overflow"};
        float* r = reinterpret_cast<float*>(base + used);
        used += bytes;
        return r;
    }
};

// activation buffers of one forward/backward with batch B on an I x I grid
struct Acts {
    float *x, *psi;
    std::vector<float*> f, upre, qpre, cdown, res, umid, cpost, tpost, qpost, uout;
    float *q1, *u1, *c2, *t2, *q2, *u2;
    // gradients
    std::vector<float*> gf, gu, t1, t2b, t3;
    float *gpsi, *gtmp;
    float *wloss, *rloss, *scr;
    float* wpart;                  // partial sums of the deterministic weight gradients
    size_t wpart_floats;
};

size_t level_elems(mgnet* n, int B, int I, int l) { return (size_t)B * n->C(l) * (I >> l) * (I >> l); }

// floats of the weight-gradient partial sums: at least every parameter once
// (one partial block of the largest layer) and 4 Mi (16 MB)
size_t wpart_floats(mgnet* n) { return n->np > ((size_t)1 << 22) ? n->np : ((size_t)1 << 22); }

Acts carve(mgnet* n, Arena& ar, int B, int I) {
    Acts a{};
    const size_t nin = (size_t)B * 2 * n->M * I * I;
    a.x = ar.f(nin);
    a.psi = ar.f(nin);
    a.gpsi = ar.f(nin);
    a.gtmp = ar.f(nin);
    a.wloss = ar.f(nin);
    a.rloss = ar.f(nin);
    a.scr = ar.f(nin);
    a.wpart_floats = wpart_floats(n);
    a.wpart = ar.f(a.wpart_floats);
    const int L = n->L;
    for (int l = 0; l < L; ++l) {
        const size_t e = level_elems(n, B, I, l);
        a.f.push_back(ar.f(e));
        a.upre.push_back(ar.f(e));
        a.qpre.push_back(ar.f(e));
        a.cdown.push_back(ar.f(e));
        a.res.push_back(ar.f(e));
        a.umid.push_back(ar.f(e));
        a.cpost.push_back(ar.f(e));
        a.tpost.push_back(ar.f(e));
        a.qpost.push_back(ar.f(e));
        a.uout.push_back(ar.f(e));
        a.gf.push_back(ar.f(e));
        a.gu.push_back(ar.f(e));
        a.t1.push_back(ar.f(e));
        a.t2b.push_back(ar.f(e));
        a.t3.push_back(ar.f(e));
    }
    const size_t e = level_elems(n, B, I, L - 1);
    a.q1 = ar.f(e);
    a.u1 = ar.f(e);
    a.c2 = ar.f(e);
    a.t2 = ar.f(e);
    a.q2 = ar.f(e);
    a.u2 = ar.f(e);
    return a;
}

size_t arena_bytes(mgnet* n, int B, int I) {
    size_t total = 7 * ((size_t)B * 2 * n->M * I * I * 4 + 256) + wpart_floats(n) * 4 + 256;
    for (int l = 0; l < n->L; ++l) total += 15 * (level_elems(n, B, I, l) * 4 + 256);
    total += 6 * (level_elems(n, B, I, n->L - 1) * 4 + 256);
    return total + 4096;
}

Acts workspace(mgnet* n, int B, int I) {
    const size_t need = arena_bytes(n, B, I);
    if (!n->ws || n->ws_bytes < need) {
        if (n->ws) cudaFree(n->ws);
        n->ws = nullptr;
        check(cudaMalloc(&n->ws, need), "cudaMalloc (network workspace)");
        n->ws_bytes = need;
    }
    Arena ar{static_cast<char*>(n->ws), 0, n->ws_bytes};
    return carve(n, ar, B, I);
}

// ------------------------------------------------------------------ conv helpers
ConvArgs cv(const float* x, int B, int Ci, int Hi, const float* w, int so, int si, int KK, int Co,
            int Hg, int S, float* y, int Ho, const Taps& tp) {
    ConvArgs a;
    a.x = x; a.B = B; a.Ci = Ci; a.Hi = Hi; a.Wi = Hi;
    a.w = w; a.so = so; a.si = si; a.KK = KK; a.Co = Co;
    a.Hg = Hg; a.Wg = Hg; a.S = S;
    a.y = y; a.Ho = Ho; a.Wo = Ho;
    a.tp = tp;
    return a;
}

WgradArgs wg(const float* g, int B, int Co, int Hg, const float* x, int Ci, int Hi, int S, float* dw,
             int so, int si, int KK, const Taps& tp) {
    WgradArgs a;
    a.g = g; a.B = B; a.Co = Co; a.Hgo = Hg; a.Wgo = Hg; a.Hg = Hg; a.Wg = Hg;
    a.x = x; a.Ci = Ci; a.Hi = Hi; a.Wi = Hi; a.S = S;
    a.dw = dw; a.so = so; a.si = si; a.KK = KK;
    a.tp = tp;
    return a;
}

// backward data of a stride-1 kxk / 1x1 convolution with weight [Co][Ci]:
// gin (Ci channels) (+)= conv(gout, flipped taps, swapped weight roles)
void bwd_data_s1(mgnet* n, const float* gout, int B, int Co, int H, const float* w, int Ci, int k,
                 float* gin, bool accumulate, const float* mask) {
    ConvArgs a = cv(gout, B, Co, H, w, 1, Ci, k * k, Ci, H, 1, gin, H, nn::taps_conv_flipped(k, k / 2));
    a.accumulate = accumulate;
    a.mask = mask;
    nn::conv(a, n->stream);
}

// ------------------------------------------------------------------ CoeffNet
// Features of more contexts than this are not kept: a server sets up a new
// context per request, and the least recently used entry (never one of the
// up to 16 samples of the current batch) makes room.
constexpr size_t kFeatureCache = 64;

Features& features(mgnet* n, rte_ctx* ctx, bool force) {
    if (n->feats.size() >= kFeatureCache && !n->feats.count(ctx->uid)) {
        auto old = n->feats.begin();
        for (auto it = n->feats.begin(); it != n->feats.end(); ++it)
            if (it->second.stamp < old->second.stamp) old = it;
        if (old->second.block) cudaFree(old->second.block);   // waits for the kernels that read it
        n->feats.erase(old);
    }
    Features& F = n->feats[ctx->uid];
    F.stamp = ++n->fclock;
    const int I = ctx->I, L = n->L;
    if (!force && F.version == n->version && F.I == I) return F;
    if (!F.block || F.I != I) {
        if (F.block) cudaFree(F.block);
        F.block = nullptr;
        size_t bytes = 0;
        for (int l = 0; l < L; ++l) {
            const size_t hw = (size_t)(I >> l) * (I >> l);
            bytes += 2 * ((size_t)n->Cc(l) * hw * 4 + 256) + 2 * (n->Cc(l) * 4 + 256) +
                     2 * ((size_t)n->C(l) * hw * 4 + 256);
        }
        check(cudaMalloc(&F.block, bytes), "cudaMalloc (CoeffNet features)");
        Arena ar{static_cast<char*>(F.block), 0, bytes};
        F.zc.clear(); F.gc.clear(); F.mean.clear(); F.inv.clear(); F.a.clear(); F.ai.clear();
        for (int l = 0; l < L; ++l) {
            const size_t hw = (size_t)(I >> l) * (I >> l);
            F.zc.push_back(ar.f(n->Cc(l) * hw));
            F.gc.push_back(ar.f(n->Cc(l) * hw));
            F.mean.push_back(ar.f(n->Cc(l)));
            F.inv.push_back(ar.f(n->Cc(l)));
            F.a.push_back(ar.f(n->C(l) * hw));
            F.ai.push_back(ar.f(n->C(l) * hw));
        }
        F.I = I;
    }
    const float* in = ctx->coef_in;
    int cin = n->cin, Hin = I;
    for (int l = 0; l < L; ++l) {
        const int H = I >> l, S = l == 0 ? 1 : 2;
        nn::conv(cv(in, 1, cin, Hin, P(n, "coef" + std::to_string(l) + ".w"), cin, 1, 9, n->Cc(l), H,
                    S, F.zc[l], H, nn::taps_conv(3, 1)), n->stream);
        nn::bn_stats(F.zc[l], 1, n->Cc(l), H * H, F.mean[l], F.inv[l], n->stream);
        nn::bn_relu(F.zc[l], 1, n->Cc(l), H * H, F.mean[l], F.inv[l],
                    P(n, "coef" + std::to_string(l) + ".gamma"), P(n, "coef" + std::to_string(l) + ".beta"),
                    F.gc[l], n->stream);
        for (int h = 0; h < 2; ++h) {
            const std::string nm = (h == 0 ? "a" : "ainv") + std::to_string(l);
            ConvArgs a = cv(F.gc[l], 1, n->Cc(l), H, P(n, nm + ".w"), n->Cc(l), 1, 1, n->C(l), H, 1,
                            h == 0 ? F.a[l] : F.ai[l], H, nn::taps_conv(1, 0));
            a.bias = P(n, nm + ".b");
            a.cst = 1.f;
            nn::conv(a, n->stream);
        }
        in = F.gc[l];
        cin = n->Cc(l);
        Hin = H;
    }
    F.version = n->version;
    return F;
}

// ------------------------------------------------------------------ forward
// FP32 forward (CUDA cores). x must already hold the normalised inputs
// [B][2M][I][I]; writes a.psi.  keep: store the pre-gate values the backward
// pass needs (training).
void forward(mgnet* n, const Features& F, Acts& a, int B, int I, bool keep) {
    const int L = n->L, M2 = 2 * n->M;
    const Taps t3 = nn::taps_conv(3, 1), t1 = nn::taps_conv(1, 0);
    auto conv = [&](const ConvArgs& c) { nn::conv(c, n->stream); };
    auto kept = [&](float* q) { return keep ? q : nullptr; };
    conv(cv(a.x, B, M2, I, P(n, "lift.w"), M2, 1, 1, n->C(0), I, 1, a.f[0], I, t1));
    auto smooth_first = [&](int l, float* q, float* u) {     // u = (B * ReLU(f)) o ainv
        const int H = I >> l, C = n->C(l);
        ConvArgs c = cv(a.f[l], B, C, H, P(n, sl("B", l)), C, 1, 9, C, H, 1, u, H, t3);
        c.relu_in = n->act; c.raw = kept(q); c.gate = F.ai[l]; c.gate_bcast = 1;
        conv(c);
    };
    auto residual = [&](int l, const float* u, float* craw, float* out) {   // f - (A * u) o a
        const int H = I >> l, C = n->C(l);
        ConvArgs c = cv(u, B, C, H, P(n, sl("A", l)), C, 1, 9, C, H, 1, out, H, t3);
        c.raw = kept(craw); c.gate = F.a[l]; c.gate_bcast = 1; c.sign = -1.f; c.base = a.f[l];
        conv(c);
    };
    auto smooth_update = [&](int l, const float* t, float* q, const float* u, float* out) {
        const int H = I >> l, C = n->C(l);
        ConvArgs c = cv(t, B, C, H, P(n, sl("B", l)), C, 1, 9, C, H, 1, out, H, t3);
        c.relu_in = n->act; c.raw = kept(q); c.gate = F.ai[l]; c.gate_bcast = 1; c.base = u;
        conv(c);
    };
    for (int l = 0; l + 1 < L; ++l) {
        const int H = I >> l;
        smooth_first(l, a.qpre[l], a.upre[l]);
        residual(l, a.upre[l], a.cdown[l], a.res[l]);
        conv(cv(a.res[l], B, n->C(l), H, P(n, sl("R", l)), n->C(l), 1, 9, n->C(l + 1), H / 2, 2,
                a.f[l + 1], H / 2, t3));
    }
    smooth_first(L - 1, a.q1, a.u1);
    residual(L - 1, a.u1, a.c2, a.t2);
    smooth_update(L - 1, a.t2, a.q2, a.u1, a.u2);
    float* uup = a.u2;
    for (int l = L - 2; l >= 0; --l) {
        const int H = I >> l;
        // u_mid = u_pre + P *^T u_coarse: each fine pixel belongs to exactly one
        // parity class, so every class adds u_pre to its own pixels
        for (int py = 0; py < 2; ++py)
            for (int px = 0; px < 2; ++px) {
                ConvArgs c = cv(uup, B, n->C(l + 1), H / 2, P(n, sl("P", l)), 1, n->C(l), 16, n->C(l),
                                H / 2, 1, a.umid[l], H, nn::taps_parity(4, py, px));
                c.OS = 2; c.OY0 = py; c.OX0 = px; c.base = a.upre[l];
                conv(c);
            }
        residual(l, a.umid[l], a.cpost[l], a.tpost[l]);
        smooth_update(l, a.tpost[l], a.qpost[l], a.umid[l], a.uout[l]);
        uup = a.uout[l];
    }
    ConvArgs c = cv(uup, B, n->C(0), I, P(n, "proj.w"), n->C(0), 1, 1, M2, I, 1, a.psi, I, t1);
    c.base = a.x;
    conv(c);
}

// ------------------------------------------------------------------ tensor-core forward
// Inference forward on the tensor cores (conv_tc.cu): the same layers as
// forward(), BF16 C8 activations, FP32 accumulation and gating.  Every layer of
// the V-cycle is linear or ReLU without bias and the gates depend on the medium
// only, so the network is positively homogeneous, rms(r) Net(r / rms(r)) =
// Net(r): the input is fed unnormalised and z = r + proj(u) is written directly.
struct TcActs {
    std::vector<void*> f, upre, res, umid, tpost, uout;
    void *u1 = nullptr, *t2 = nullptr, *u2 = nullptr;
};

size_t c8_bytes(int C, int H) { return (((size_t)(C + 7) / 8) * H * H * 16 + 255) & ~(size_t)255; }

TcActs tc_workspace(mgnet* n, int I, int B) {
    const int L = n->L;
    size_t need = 0;
    for (int l = 0; l < L; ++l) need += 6 * B * c8_bytes(n->C(l), I >> l);
    need += 3 * B * c8_bytes(n->C(L - 1), I >> (L - 1));
    if (!n->tc_ws || n->tc_ws_bytes < need) {
        if (n->tc_ws) cudaFree(n->tc_ws);
        n->tc_ws = nullptr;
        check(cudaMalloc(&n->tc_ws, need), "cudaMalloc (tensor-core workspace)");
        n->tc_ws_bytes = need;
    }
    char* p = static_cast<char*>(n->tc_ws);
    auto take = [&](int C, int H) { void* r = p; p += B * c8_bytes(C, H); return r; };
    TcActs A;
    for (int l = 0; l < L; ++l) {
        const int C = n->C(l), H = I >> l;
        A.f.push_back(take(C, H));
        A.upre.push_back(take(C, H));
        A.res.push_back(take(C, H));
        A.umid.push_back(take(C, H));
        A.tpost.push_back(take(C, H));
        A.uout.push_back(take(C, H));
    }
    const int C = n->C(L - 1), H = I >> (L - 1);
    A.u1 = take(C, H);
    A.t2 = take(C, H);
    A.u2 = take(C, H);
    return A;
}

enum class TcMode { Plan, Pack, Run };

// The samples of one tensor-core forward: B solves of one grid size, each
// with its input r, output z and medium (features F).
struct TcSamples {
    int B = 1;
    const Features* F[nn::kTcMaxBatch] = {};
    const double* r[nn::kTcMaxBatch] = {};
    const float* r32[nn::kTcMaxBatch] = {};    // FP32 inputs instead of r (all samples or none)
    float* z[nn::kTcMaxBatch] = {};
};

// Plan: returns the packed-weight bytes; Pack: packs then runs; Run: runs.
// Every sample's output is the same bits as a forward of it alone.
size_t tc_forward(mgnet* n, const TcSamples& S, int I, TcMode mode) {
    const int L = n->L, M2 = 2 * n->M, B = S.B;
    const Taps t3 = nn::taps_conv(3, 1), t1 = nn::taps_conv(1, 0);
    TcActs A;
    if (mode != TcMode::Plan) A = tc_workspace(n, I, B);
    auto gates = [&](nn::TcConv& c, int l, bool inverse) {
        for (int b = 0; b < B; ++b)
            c.gate_b[b] = S.F[b] ? (inverse ? S.F[b]->ai[l] : S.F[b]->a[l]) : nullptr;
    };
    size_t cursor = 0;
    auto run = [&](nn::TcConv c, const char* wname, int so, int si, int KK, const Taps& tp) {
        const size_t bytes = nn::tc_weight_bytes(tp.T, c.classes, c.Ci, c.Co);
        void* dst = static_cast<char*>(n->tcw) + cursor;
        cursor += bytes;
        if (mode == TcMode::Plan) return;
        if (mode == TcMode::Pack) nn::tc_pack(P(n, wname), so, si, KK, tp, c.classes, c.Ci, c.Co, dst, n->stream);
        c.w = dst;
        c.T = tp.T / c.classes;
        for (int t = 0; t < tp.T; ++t) {
            c.dy[t] = tp.dy[t];
            c.dx[t] = tp.dx[t];
        }
        nn::tc_conv(c, mode == TcMode::Run, n->stream);
    };
    auto conv = [&](const void* x8, int Ci, int Hi, int Co, int Hg, int stride, void* y8, int Ho) {
        nn::TcConv c;
        c.x8 = x8; c.B = B; c.Ci = Ci; c.Hi = Hi; c.Wi = Hi;
        c.Co = Co; c.Hg = Hg; c.Wg = Hg; c.S = stride;
        c.y8 = y8; c.Ho = Ho; c.Wo = Ho;
        c.batched = 1;
        return c;
    };
    {   // lift: FP64 Krylov vectors -> f_0
        nn::TcConv c = conv(nullptr, M2, I, n->C(0), I, 1, A.f.empty() ? nullptr : A.f[0], I);
        for (int b = 0; b < B; ++b) {
            if (S.r32[0])
                c.x32_b[b] = S.r32[b];
            else
                c.x64_b[b] = S.r[b];
        }
        run(c, "lift.w", M2, 1, 1, t1);
    }
    auto smooth_first = [&](int l, void* u) {            // u = (B * act(f)) o ainv
        const int H = I >> l, C = n->C(l);
        nn::TcConv c = conv(A.f.empty() ? nullptr : A.f[l], C, H, C, H, 1, u, H);
        c.relu_in = n->act;
        gates(c, l, true);
        run(c, sl("B", l).c_str(), C, 1, 9, t3);
    };
    auto residual = [&](int l, const void* u, void* out) {   // f - (A * u) o a
        const int H = I >> l, C = n->C(l);
        nn::TcConv c = conv(u, C, H, C, H, 1, out, H);
        gates(c, l, false);
        c.sign = -1.f;
        c.base8 = A.f.empty() ? nullptr : A.f[l];
        run(c, sl("A", l).c_str(), C, 1, 9, t3);
    };
    auto smooth_update = [&](int l, const void* t, const void* u, void* out) {   // u + (B * act(t)) o ainv
        const int H = I >> l, C = n->C(l);
        nn::TcConv c = conv(t, C, H, C, H, 1, out, H);
        c.relu_in = n->act;
        gates(c, l, true);
        c.base8 = u;
        run(c, sl("B", l).c_str(), C, 1, 9, t3);
    };
    auto at = [&](std::vector<void*>& v, int l) { return v.empty() ? nullptr : v[l]; };
    for (int l = 0; l + 1 < L; ++l) {
        const int H = I >> l;
        smooth_first(l, at(A.upre, l));
        residual(l, at(A.upre, l), at(A.res, l));
        run(conv(at(A.res, l), n->C(l), H, n->C(l + 1), H / 2, 2, at(A.f, l + 1), H / 2), sl("R", l).c_str(),
            n->C(l), 1, 9, t3);
    }
    smooth_first(L - 1, A.u1);
    residual(L - 1, A.u1, A.t2);
    smooth_update(L - 1, A.t2, A.u1, A.u2);
    const void* uup = A.u2;
    for (int l = L - 2; l >= 0; --l) {
        const int H = I >> l;
        {   // u_mid = u_pre + P *^T u_coarse: the four parity classes in one launch
            nn::TcConv c = conv(uup, n->C(l + 1), H / 2, n->C(l), H / 2, 1, at(A.umid, l), H);
            c.OS = 2;
            c.classes = 4;
            c.base8 = at(A.upre, l);
            Taps all{};
            for (int q = 0; q < 4; ++q) {
                const Taps tq = nn::taps_parity(4, q / 2, q % 2);
                c.oy0[q] = q / 2;
                c.ox0[q] = q % 2;
                for (int t = 0; t < tq.T; ++t) {
                    all.dy[all.T] = tq.dy[t];
                    all.dx[all.T] = tq.dx[t];
                    all.wi[all.T] = tq.wi[t];
                    ++all.T;
                }
            }
            all.finish();
            run(c, sl("P", l).c_str(), 1, n->C(l), 16, all);
        }
        residual(l, at(A.umid, l), at(A.tpost, l));
        smooth_update(l, at(A.tpost, l), at(A.umid, l), at(A.uout, l));
        uup = at(A.uout, l);
    }
    {   // z = r + proj(u_0), FP32 [2M][I][I]
        nn::TcConv c = conv(uup, n->C(0), I, M2, I, 1, nullptr, I);
        for (int b = 0; b < B; ++b) {
            c.y32_b[b] = S.z[b];
            if (S.r32[0])
                c.base32_b[b] = S.r32[b];
            else
                c.base64_b[b] = S.r[b];
        }
        run(c, "proj.w", n->C(0), 1, 1, t1);
    }
    return cursor;
}

void tc_precondition(mgnet* n, const TcSamples& S, int I) {
    if (n->tcw_version != n->version) {
        const size_t need = tc_forward(n, TcSamples{}, I, TcMode::Plan);
        if (!n->tcw || n->tcw_bytes < need) {
            if (n->tcw) cudaFree(n->tcw);
            n->tcw = nullptr;
            check(cudaMalloc(&n->tcw, need), "cudaMalloc (packed weights)");
            n->tcw_bytes = need;
        }
        tc_forward(n, S, I, TcMode::Pack);
        n->tcw_version = n->version;
    } else {
        tc_forward(n, S, I, TcMode::Run);
    }
}

// ------------------------------------------------------------------ backward
// Given a.gpsi (dLoss/dpsi), accumulate every parameter gradient into n->g.
void backward(mgnet* n, Features& F, Acts& a, rte_ctx* ctx, int B, int I) {
    nn::WgradScratch wscr{a.wpart, a.wpart_floats, ctx->num_sms};
    struct ResetScratch {
        ~ResetScratch() { nn::tl_wgrad_scratch = nullptr; }
    } reset_scratch;
    nn::tl_wgrad_scratch = &wscr;
    const int L = n->L, M2 = 2 * n->M;
    const Taps t3 = nn::taps_conv(3, 1), t1 = nn::taps_conv(1, 0), t4 = nn::taps_conv(4, 1);
    cudaStream_t st = n->stream;
    std::vector<float*> ga(L), gai(L);
    // gate gradients per level live in the t3 scratch of the level (size >= C H^2)
    for (int l = 0; l < L; ++l) {
        const size_t e = level_elems(n, B, I, l);
        check(cudaMemsetAsync(a.gf[l], 0, e * 4, st), "memset");
        ga[l] = a.t3[l];
        gai[l] = a.t3[l] + (size_t)n->C(l) * (I >> l) * (I >> l);
        check(cudaMemsetAsync(ga[l], 0, (size_t)2 * n->C(l) * (I >> l) * (I >> l) * 4, st), "memset");
    }
    (void)ctx;
    // psi = x + proj * u_out0
    const float* u0 = L > 1 ? a.uout[0] : a.u2;
    nn::wgrad(wg(a.gpsi, B, M2, I, u0, n->C(0), I, 1, G(n, "proj.w"), n->C(0), 1, 1, t1), st);
    float* gu_up = a.gu[0];      // gradient of the current level's output u
    {
        ConvArgs c = cv(a.gpsi, B, M2, I, P(n, "proj.w"), 1, n->C(0), 1, n->C(0), I, 1, gu_up, I, t1);
        nn::conv(c, st);
    }
    // smoothing-step backward: u_out = u_in + (B * ReLU(t)) o ai ; t = f - (A * u_in) o a
    // gu: gradient of u_out on entry, of u_in on exit (in place); t stored, q raw stored
    auto smooth_bwd = [&](int l, float* gu, const float* t, const float* q, const float* c,
                          const float* u_in, bool has_A) {
        const int H = I >> l, C = n->C(l);
        const size_t chw = (size_t)C * H * H;
        float* gq = a.t1[l];
        float* gt = a.t2b[l];
        nn::gate_bwd(gu, F.ai[l], q, 1.f, B, chw, gq, gai[l], st);
        // gt = bwd_data(B_l, gq) (masked by t > 0 for ReLU) ; dB += wgrad(gq, act(t))
        bwd_data_s1(n, gq, B, C, H, P(n, sl("B", l)), C, 3, gt, false, n->act ? t : nullptr);
        {
            WgradArgs w = wg(gq, B, C, H, t, C, H, 1, G(n, sl("B", l)), C, 1, 9, t3);
            w.relu_in = n->act;
            nn::wgrad(w, st);
        }
        nn::axpy(a.gf[l], gt, 1.f, (size_t)B * chw, st);
        if (!has_A) return;
        // t = f - c o a: gc = -gt o a ; ga += -gt o c
        float* gc = a.t1[l];
        nn::gate_bwd(gt, F.a[l], c, -1.f, B, chw, gc, ga[l], st);
        bwd_data_s1(n, gc, B, C, H, P(n, sl("A", l)), C, 3, gu, true, nullptr);
        nn::wgrad(wg(gc, B, C, H, u_in, C, H, 1, G(n, sl("A", l)), C, 1, 9, t3), st);
    };
    // up path, reversed: levels 0 .. L-2
    for (int l = 0; l + 1 < L; ++l) {
        const int H = I >> l, C = n->C(l), Cn = n->C(l + 1);
        // post-smoothing at level l (input umid, t = tpost, q = qpost, c = cpost)
        smooth_bwd(l, gu_up, a.tpost[l], a.qpost[l], a.cpost[l], a.umid[l], true);
        // umid = upre + P^T-conv(u_{l+1}): g_upre = g_umid (kept in gu[l]);
        // g_u_{l+1} = conv4x4 s2 of g_umid with P ; dP += wgrad
        float* gnext = a.gu[l + 1];
        const float* ucoarse = (l + 1 == L - 1) ? a.u2 : a.uout[l + 1];
        nn::conv(cv(gu_up, B, C, H, P(n, sl("P", l)), C, 1, 16, Cn, H / 2, 2, gnext, H / 2, t4), st);
        nn::wgrad(wg(ucoarse, B, Cn, H / 2, gu_up, C, H, 2, G(n, sl("P", l)), C, 1, 16, t4), st);
        gu_up = gnext;
    }
    // coarsest: u2 = u1 + (B * ReLU(t2)) o ai ; t2 = f - (A * u1) o a ; u1 = (B * ReLU(f)) o ai
    {
        const int l = L - 1;
        smooth_bwd(l, gu_up, a.t2, a.q2, a.c2, a.u1, true);
        smooth_bwd(l, gu_up, a.f[l], a.q1, nullptr, nullptr, false);
    }
    // down path, reversed: levels L-2 .. 0; a.gu[l] holds g_umid == g_upre
    for (int l = L - 2; l >= 0; --l) {
        const int H = I >> l, C = n->C(l), Cn = n->C(l + 1);
        // restriction f_{l+1} = R *s2 res: g_res = bwd data (parity classes) ; dR += wgrad
        float* gres = a.t2b[l];
        for (int py = 0; py < 2; ++py)
            for (int px = 0; px < 2; ++px) {
                ConvArgs c = cv(a.gf[l + 1], B, Cn, H / 2, P(n, sl("R", l)), 1, C, 9, C, H / 2, 1, gres, H,
                                nn::taps_parity(3, py, px));
                c.OS = 2; c.OY0 = py; c.OX0 = px;
                nn::conv(c, st);
            }
        nn::wgrad(wg(a.gf[l + 1], B, Cn, H / 2, a.res[l], C, H, 2, G(n, sl("R", l)), C, 1, 9, t3), st);
        // res = f - (A * upre) o a
        const size_t chw = (size_t)C * H * H;
        nn::axpy(a.gf[l], gres, 1.f, (size_t)B * chw, st);
        float* gc = a.t1[l];
        nn::gate_bwd(gres, F.a[l], a.cdown[l], -1.f, B, chw, gc, ga[l], st);
        bwd_data_s1(n, gc, B, C, H, P(n, sl("A", l)), C, 3, a.gu[l], true, nullptr);
        nn::wgrad(wg(gc, B, C, H, a.upre[l], C, H, 1, G(n, sl("A", l)), C, 1, 9, t3), st);
        // upre = (B * ReLU(f)) o ai
        smooth_bwd(l, a.gu[l], a.f[l], a.qpre[l], nullptr, nullptr, false);
    }
    // lift: f0 = lift * x
    nn::wgrad(wg(a.gf[0], B, n->C(0), I, a.x, M2, I, 1, G(n, "lift.w"), M2, 1, 1, t1), st);
    // CoeffNet: heads, then BN-ReLU and convolutions from the top level down
    std::vector<float*> ggc(L);
    for (int l = 0; l < L; ++l) {
        const int H = I >> l;
        ggc[l] = a.t2b[l];          // scratch of size >= Cc H^2 (batch 1)
        check(cudaMemsetAsync(ggc[l], 0, (size_t)n->Cc(l) * H * H * 4, st), "memset");
        for (int h = 0; h < 2; ++h) {
            const std::string nm = (h == 0 ? "a" : "ainv") + std::to_string(l);
            const float* gg = h == 0 ? ga[l] : gai[l];
            ConvArgs c = cv(gg, 1, n->C(l), H, P(n, nm + ".w"), 1, n->Cc(l), 1, n->Cc(l), H, 1, ggc[l], H, t1);
            c.accumulate = 1;
            nn::conv(c, st);
            nn::wgrad(wg(gg, 1, n->C(l), H, F.gc[l], n->Cc(l), H, 1, G(n, nm + ".w"), n->Cc(l), 1, 1, t1), st);
            nn::channel_sum(gg, 1, n->C(l), H * H, G(n, nm + ".b"), st);
        }
    }
    for (int l = L - 1; l >= 0; --l) {
        const int H = I >> l;
        float* gz = a.t1[l];
        nn::bn_relu_bwd(F.zc[l], F.gc[l], ggc[l], 1, n->Cc(l), H * H, F.mean[l], F.inv[l],
                        P(n, "coef" + std::to_string(l) + ".gamma"),
                        G(n, "coef" + std::to_string(l) + ".gamma"),
                        G(n, "coef" + std::to_string(l) + ".beta"), gz, st);
        const float* xin = l == 0 ? ctx->coef_in : F.gc[l - 1];
        const int cin = l == 0 ? n->cin : n->Cc(l - 1);
        const int Hin = l == 0 ? I : (I >> (l - 1));
        const int S = l == 0 ? 1 : 2;
        nn::wgrad(wg(gz, 1, n->Cc(l), H, xin, cin, Hin, S, G(n, "coef" + std::to_string(l) + ".w"), cin, 1, 9, t3), st);
        if (l > 0) {
            for (int py = 0; py < 2; ++py)
                for (int px = 0; px < 2; ++px) {
                    ConvArgs c = cv(gz, 1, n->Cc(l), H, P(n, "coef" + std::to_string(l) + ".w"), 1, cin, 9, cin,
                                    H, 1, ggc[l - 1], Hin, nn::taps_parity(3, py, px));
                    c.OS = 2; c.OY0 = py; c.OX0 = px; c.accumulate = 1;
                    nn::conv(c, st);
                }
        }
    }
}

// ------------------------------------------------------------------ glue kernels
// x[b] = r_b * sqrt(n) / ||r_b|| as float (norms in scal[b])
__global__ void k_normalise_in(const double* __restrict__ r, int64_t n, const double* __restrict__ nrm,
                               float* __restrict__ x) {
    const double s = nrm[0] > 0.0 ? sqrt((double)n) / nrm[0] : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = (float)(r[i] * s);
}

__global__ void k_scale_out(const float* __restrict__ psi, int64_t n, const double* __restrict__ nrm,
                            float* __restrict__ z) {
    const float s = (float)(nrm[0] / sqrt((double)n));
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        z[i] = psi[i] * s;
}

// Block partial sums of the loss norms, added in a fixed order by k_finish_pairs
// (no atomics: the loss and its gradient are the same bits on every run).
// part[2 blockIdx.x + {0, 1}] = the block's sums of a^2 and b^2 (float inputs,
// double sums)
__global__ void k_norms2(const float* __restrict__ a, const float* __restrict__ b, int64_t n,
                         double* __restrict__ part) {
    __shared__ double ra[32], rb[32];
    double sa = 0.0, sb = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        sa += (double)a[i] * a[i];
        sb += (double)b[i] * b[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_down_sync(0xffffffffu, sa, o);
        sb += __shfl_down_sync(0xffffffffu, sb, o);
    }
    if ((threadIdx.x & 31) == 0) { ra[threadIdx.x >> 5] = sa; rb[threadIdx.x >> 5] = sb; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { ta += ra[w]; tb += rb[w]; }
        part[2 * blockIdx.x] = ta;
        part[2 * blockIdx.x + 1] = tb;
    }
}

// out[k] += sum over blocks b < nb of part[width b + k], k < width (one block
// of 256 threads; fixed summation order)
__global__ void k_finish_pairs(const double* __restrict__ part, int nb, int width, double* __restrict__ out) {
    __shared__ double red[256];
    for (int k = 0; k < width; ++k) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[(size_t)width * b + k];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int h = blockDim.x / 2; h > 0; h >>= 1) {
            if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] += red[0];
        __syncthreads();
    }
}

// y = (float) (s x)
__global__ void k_scale_to_f(const double* __restrict__ x, double s, float* __restrict__ y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)(s * x[i]);
}

// y -= x
__global__ void k_sub_from_d(double* __restrict__ y, const float* __restrict__ x, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] -= (double)x[i];
}

// part[2 blockIdx.x + {0, 1}] = the block's ||a||^2 (double) and ||b||^2 (float)
__global__ void k_sumsq_df(const double* __restrict__ a, int64_t na, const float* __restrict__ b, int64_t nb,
                           double* __restrict__ part) {
    __shared__ double ra[32], rb[32];
    double sa = 0.0, sb = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < na; i += stride) sa = fma(a[i], a[i], sa);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += stride)
        sb += (double)b[i] * b[i];
    for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_down_sync(0xffffffffu, sa, o);
        sb += __shfl_down_sync(0xffffffffu, sb, o);
    }
    if ((threadIdx.x & 31) == 0) { ra[threadIdx.x >> 5] = sa; rb[threadIdx.x >> 5] = sb; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { ta += ra[w]; tb += rb[w]; }
        part[2 * blockIdx.x] = ta;
        part[2 * blockIdx.x + 1] = tb;
    }
}

__global__ void k_sub_f(const float* __restrict__ a, const float* __restrict__ b, int64_t n,
                        float* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] - b[i];
}

// part[blockIdx.x] = the block's sum of r^2
__global__ void k_double_norm(const double* __restrict__ r, int64_t n, double* __restrict__ part) {
    __shared__ double red[32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += r[i] * r[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

__global__ void k_sqrt_inplace(double* v, int count) {
    if (threadIdx.x < count) v[threadIdx.x] = sqrt(v[threadIdx.x]);
}

int grid_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    return (int)(b < 2048 ? (b > 0 ? b : 1) : 2048);
}

// The network works on the stream of the context it is called with.
void check_ctx(mgnet* n, rte_ctx* ctx) {
    if (ctx->M != n->M) throw StatusError{RTE_EINVAL, "network and context have different M"};
    if (ctx->I % (1 << (n->L - 1)) != 0 || (ctx->I >> (n->L - 1)) < 1)
        throw StatusError{RTE_EINVAL, "I must be divisible by 2^(levels-1)"};
    if (ctx->stream != n->stream) n->stream = ctx->stream;
}

// normalise a batch of FP64 right-hand sides into a.x; norms into n->d_scal[b]
void load_inputs(mgnet* n, rte_ctx* ctx, const double* const* r, int B, Acts& a) {
    const int64_t len = ctx->n;
    check(cudaMemsetAsync(n->d_scal, 0, 64 * sizeof(double), n->stream), "memset");
    for (int b = 0; b < B; ++b) {
        k_double_norm<<<grid_for(len), 256, 0, n->stream>>>(r[b], len, n->d_part);
        k_finish_pairs<<<1, 256, 0, n->stream>>>(n->d_part, grid_for(len), 1, n->d_scal + b);
    }
    k_sqrt_inplace<<<1, 64, 0, n->stream>>>(n->d_scal, B);
    for (int b = 0; b < B; ++b)
        k_normalise_in<<<grid_for(len), 256, 0, n->stream>>>(r[b], len, n->d_scal + b, a.x + (size_t)b * len);
    check(cudaGetLastError(), "load_inputs");
}

// Eq. loss_delta: loss = mean_b ||F (A (mask o D psi_b) - x_b)|| / ||x_b||, A in
// FP64; a.gpsi = its gradient D^T (mask o A^T F^T res_b) / (||res_b|| ||x_b|| B).
double loss_and_seed_filtered(mgnet* n, rte_ctx* ctx, Acts& a, int B) {
    const int64_t len = ctx->n, R = atfps_rows(ctx);
    if (R < 0) throw StatusError{RTE_EINVAL, "the filtered loss needs rte_atfps_setup on the context"};
    const size_t need = (4 * (size_t)len + (size_t)B * (R + 1)) * sizeof(double) + 1024;
    if (!n->lscr || n->lscr_bytes < need) {
        if (n->lscr) cudaFree(n->lscr);
        n->lscr = nullptr;
        check(cudaMalloc(&n->lscr, need), "cudaMalloc (filtered loss scratch)");
        n->lscr_bytes = need;
    }
    double* alpha = static_cast<double*>(n->lscr);
    double* y = alpha + len;
    double* u = y + len;
    double* galpha = u + len;
    double* res = galpha + len;          // [B][R]
    double* sums = n->d_scal + 32;
    check(cudaMemsetAsync(sums, 0, 2 * B * sizeof(double), n->stream), "memset");
    for (int b = 0; b < B; ++b) {
        const float* psi = a.psi + (size_t)b * len;
        const float* x = a.x + (size_t)b * len;
        launch_block_apply(ctx, false, psi, false, alpha, true);            // D psi
        atfps_mask_mul(ctx, alpha);                                          // D_delta psi
        launch_apply(ctx, true, alpha, y, true, nullptr);                   // A alpha
        k_sub_from_d<<<grid_for(len), 256, 0, n->stream>>>(y, x, len);
        atfps_apply(ctx, y, res + (size_t)b * R);
        k_sumsq_df<<<grid_for(len), 256, 0, n->stream>>>(res + (size_t)b * R, R, x, len, n->d_part);
        k_finish_pairs<<<1, 256, 0, n->stream>>>(n->d_part, grid_for(len), 2, sums + 2 * b);
    }
    check(cudaGetLastError(), "filtered loss");
    check(cudaMemcpyAsync(n->h_scal, sums, 2 * B * sizeof(double), cudaMemcpyDeviceToHost, n->stream), "d2h");
    check(cudaStreamSynchronize(n->stream), "sync");
    double loss = 0.0;
    for (int b = 0; b < B; ++b) {
        const double nr = std::sqrt(n->h_scal[2 * b]), nx = std::sqrt(n->h_scal[2 * b + 1]);
        loss += nr / nx / B;
        float* g = a.gpsi + (size_t)b * len;
        atfps_apply_t(ctx, res + (size_t)b * R, u);                          // F^T res
        launch_apply_adjoint(ctx, true, u, galpha);                          // A^T
        atfps_mask_mul(ctx, galpha);
        launch_block_apply(ctx, true, galpha, true, alpha, true);            // D^T
        k_scale_to_f<<<grid_for(len), 256, 0, n->stream>>>(alpha, nr > 0 ? 1.0 / (nr * nx * B) : 0.0, g, len);
        check(cudaGetLastError(), "k_scale_to_f");
    }
    return loss;
}

// loss = mean_b ||x_b - B psi_b|| / ||x_b|| ; a.gpsi = its gradient
double loss_and_seed(mgnet* n, rte_ctx* ctx, Acts& a, int B) {
    if (n->loss == MGNET_LOSS_FILTERED) return loss_and_seed_filtered(n, ctx, a, B);
    const int64_t len = ctx->n;
    double* sums = n->d_scal + 32;
    check(cudaMemsetAsync(sums, 0, 2 * B * sizeof(double), n->stream), "memset");
    for (int b = 0; b < B; ++b) {
        const float* psi = a.psi + (size_t)b * len;
        const float* x = a.x + (size_t)b * len;
        launch_response_apply(ctx, psi, false, a.wloss, false);            // B psi
        k_sub_f<<<grid_for(len), 256, 0, n->stream>>>(x, a.wloss, len, a.rloss + 0);
        k_norms2<<<grid_for(len), 256, 0, n->stream>>>(a.rloss, x, len, n->d_part);
        k_finish_pairs<<<1, 256, 0, n->stream>>>(n->d_part, grid_for(len), 2, sums + 2 * b);
        launch_response_apply_t(ctx, a.rloss, a.gpsi + (size_t)b * len, a.scr);   // B^T res
    }
    check(cudaMemcpyAsync(n->h_scal, sums, 2 * B * sizeof(double), cudaMemcpyDeviceToHost, n->stream), "d2h");
    check(cudaStreamSynchronize(n->stream), "sync");
    double loss = 0.0;
    for (int b = 0; b < B; ++b) {
        const double nr = std::sqrt(n->h_scal[2 * b]), nx = std::sqrt(n->h_scal[2 * b + 1]);
        loss += nr / nx / B;
        const float scale = (float)(nr > 0 ? -1.0 / (nr * nx * B) : 0.0);
        nn::scale_copy(a.gpsi + (size_t)b * len, a.gpsi + (size_t)b * len, scale, len, n->stream);
    }
    return loss;
}

}  // namespace

// ------------------------------------------------------------------ solver hooks
void mgnet_prepare(mgnet* net, rte_ctx* ctx) {
    check_ctx(net, ctx);
    features(net, ctx, false);
}

void mgnet_precondition(mgnet* net, rte_ctx* ctx, const double* v, float* z) {
    NvtxRange range("MgNet V-cycle");
    check_ctx(net, ctx);
    Features& F = features(net, ctx, false);
    // count the forward's convolutions (launches, FP32 flops) for the profile
    nn::Counters cnt;
    struct Reset {
        ~Reset() { nn::tl_counters = nullptr; }
    } reset;
    nn::tl_counters = &cnt;
    if (net->prec == MGNET_BF16) {
        ProfScope ps(ctx, K_MGNET, (double)ctx->n * 12, 0);
        TcSamples S;
        S.F[0] = &F;
        S.r[0] = v;
        S.z[0] = z;
        tc_precondition(net, S, ctx->I);
    } else {
        ProfScope ps(ctx, K_MGNET, (double)ctx->n * 12, 0);
        Acts a = workspace(net, 2, ctx->I);
        const double* rv[1] = {v};
        load_inputs(net, ctx, rv, 1, a);
        forward(net, F, a, 1, ctx->I, false);
        k_scale_out<<<grid_for(ctx->n), 256, 0, net->stream>>>(a.psi, ctx->n, net->d_scal, z);
        check(cudaGetLastError(), "k_scale_out");
        cnt.launches += 4;                                // norm, sqrt, normalise, scale
    }
    if (net->fault == MGNET_FAULT_NAN)
        check(cudaMemsetAsync(z, 0xFF, (size_t)ctx->n * sizeof(float), net->stream), "fault injection");
    ctx->prof.launches[K_MGNET] += cnt.launches;
    ctx->prof.flops[K_MGNET] += cnt.flops;
}

void mgnet_precondition_batch(mgnet* net, rte_ctx* const* ctxs, const double* const* v, float* const* z, int B) {
    if (B == 1 || net->prec != MGNET_BF16) {
        for (int b = 0; b < B; ++b) mgnet_precondition(net, ctxs[b], v[b], z[b]);
        return;
    }
    const int I = ctxs[0]->I;
    for (int b = 0; b < B; ++b) {
        check_ctx(net, ctxs[b]);
        if (ctxs[b]->I != I) throw StatusError{RTE_EINVAL, "batched preconditioning needs one grid size"};
    }
    for (int b0 = 0; b0 < B; b0 += nn::kTcMaxBatch) {
        TcSamples S;
        S.B = B - b0 < nn::kTcMaxBatch ? B - b0 : nn::kTcMaxBatch;
        for (int b = 0; b < S.B; ++b) {
            S.F[b] = &features(net, ctxs[b0 + b], false);
            S.r[b] = v[b0 + b];
            S.z[b] = z[b0 + b];
        }
        ProfScope ps(ctxs[b0], K_MGNET, (double)ctxs[b0]->n * 12 * S.B, 0);
        tc_precondition(net, S, I);
        if (net->fault == MGNET_FAULT_NAN)
            for (int b = 0; b < S.B; ++b)
                check(cudaMemsetAsync(S.z[b], 0xFF, (size_t)ctxs[b0 + b]->n * sizeof(float), net->stream),
                      "fault injection");
    }
}

__global__ void k_f32_to_f64(const float* __restrict__ x, int64_t n, double* __restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (double)x[i];
}

void mgnet_precondition_f(mgnet* net, rte_ctx* ctx, const float* v, float* z) {
    if (net->prec != MGNET_BF16) {
        // the CUDA-core forward normalises an FP64 input: widen v first
        if (net->fin64_n < (size_t)ctx->n) {
            if (net->fin64) cudaFree(net->fin64);
            net->fin64 = nullptr;
            net->fin64_n = 0;
            check(cudaMalloc(&net->fin64, (size_t)ctx->n * sizeof(double)), "cudaMalloc (network input)");
            net->fin64_n = (size_t)ctx->n;
        }
        k_f32_to_f64<<<grid_for(ctx->n), 256, 0, ctx->stream>>>(v, ctx->n, net->fin64);
        check(cudaGetLastError(), "k_f32_to_f64");
        mgnet_precondition(net, ctx, net->fin64, z);
        return;
    }
    NvtxRange range("MgNet V-cycle");
    check_ctx(net, ctx);
    Features& F = features(net, ctx, false);
    nn::Counters cnt;
    struct Reset {
        ~Reset() { nn::tl_counters = nullptr; }
    } reset;
    nn::tl_counters = &cnt;
    {
        ProfScope ps(ctx, K_MGNET, (double)ctx->n * 8, 0);
        TcSamples S;
        S.F[0] = &F;
        S.r32[0] = v;
        S.z[0] = z;
        tc_precondition(net, S, ctx->I);
    }
    if (net->fault == MGNET_FAULT_NAN)
        check(cudaMemsetAsync(z, 0xFF, (size_t)ctx->n * sizeof(float), net->stream), "fault injection");
    ctx->prof.launches[K_MGNET] += cnt.launches;
    ctx->prof.flops[K_MGNET] += cnt.flops;
}

void mgnet_precondition_batch_f(mgnet* net, rte_ctx* const* ctxs, const float* const* v, float* const* z, int B) {
    if (B == 1 || net->prec != MGNET_BF16) {
        for (int b = 0; b < B; ++b) mgnet_precondition_f(net, ctxs[b], v[b], z[b]);
        return;
    }
    const int I = ctxs[0]->I;
    for (int b = 0; b < B; ++b) {
        check_ctx(net, ctxs[b]);
        if (ctxs[b]->I != I) throw StatusError{RTE_EINVAL, "batched preconditioning needs one grid size"};
    }
    for (int b0 = 0; b0 < B; b0 += nn::kTcMaxBatch) {
        TcSamples S;
        S.B = B - b0 < nn::kTcMaxBatch ? B - b0 : nn::kTcMaxBatch;
        for (int b = 0; b < S.B; ++b) {
            S.F[b] = &features(net, ctxs[b0 + b], false);
            S.r32[b] = v[b0 + b];
            S.z[b] = z[b0 + b];
        }
        ProfScope ps(ctxs[b0], K_MGNET, (double)ctxs[b0]->n * 8 * S.B, 0);
        tc_precondition(net, S, I);
        if (net->fault == MGNET_FAULT_NAN)
            for (int b = 0; b < S.B; ++b)
                check(cudaMemsetAsync(S.z[b], 0xFF, (size_t)ctxs[b0 + b]->n * sizeof(float), net->stream),
                      "fault injection");
    }
}

}  // namespace rte

using namespace rte;

#define MG_GUARD_BEGIN try {
#define MG_GUARD_END(net)                                                                        \
    }                                                                                            \
    catch (const CudaError& e) { rte_status s = cuda_status(nullptr, e.code, e.where); if (net) net->err = rte_last_error(nullptr); return s; } \
    catch (const StatusError& e) { set_error(nullptr, e.msg); if (net) net->err = e.msg; return e.code; } \
    catch (const std::bad_alloc&) { set_error(nullptr, "host allocation failed"); return RTE_ENOMEM; } \
    catch (const std::out_of_range&) { set_error(nullptr, "unknown parameter"); return RTE_EINVAL; }

extern "C" {

RTE_API rte_status mgnet_create(const mgnet_config* cfg, void* stream, mgnet** out) {
    if (!cfg || !out) { set_error(nullptr, "NULL argument"); return RTE_EINVAL; }
    *out = nullptr;
    if (cfg->M < 4 || cfg->M % 4 || cfg->levels < 1 || cfg->levels > 8 || cfg->c0 < 1 || cfg->cmax < cfg->c0 ||
        cfg->cc < 1 || cfg->ccmax < cfg->cc || cfg->cc > cfg->c0 || cfg->ccmax > cfg->cmax ||
        (cfg->act != 0 && cfg->act != 1)) {
        set_error(nullptr, "bad network configuration (need cc <= c0, ccmax <= cmax)");
        return RTE_EINVAL;
    }
    mgnet* n = new (std::nothrow) mgnet();
    if (!n) { set_error(nullptr, "host allocation failed"); return RTE_ENOMEM; }
    n->M = cfg->M; n->L = cfg->levels; n->c0 = cfg->c0; n->cmax = cfg->cmax;
    n->cc = cfg->cc; n->ccmax = cfg->ccmax; n->act = cfg->act;
    n->stream = static_cast<cudaStream_t>(stream);
    MG_GUARD_BEGIN
    build_params(n);
    check(cudaMalloc(&n->p, n->np * 4 * 4), "cudaMalloc (parameters)");
    n->g = n->p + n->np;
    n->m = n->g + n->np;
    n->v = n->m + n->np;
    check(cudaMemsetAsync(n->p, 0, n->np * 16, n->stream), "memset");
    check(cudaMalloc(&n->d_scal, (128 + 2 * 2048) * sizeof(double)), "cudaMalloc");
    n->d_part = n->d_scal + 128;
    check(cudaMallocHost(&n->h_scal, 128 * sizeof(double)), "cudaMallocHost");
    check(cudaStreamSynchronize(n->stream), "sync");
    *out = n;
    return RTE_OK;
    }
    catch (...) {
        mgnet_destroy(n);
        set_error(nullptr, "mgnet_create failed");
        return RTE_ENOMEM;
    }
}

RTE_API rte_status mgnet_clone(const mgnet* src, void* stream, mgnet** out) {
    if (!src || !out) { set_error(nullptr, "NULL argument"); return RTE_EINVAL; }
    mgnet_config cfg{src->M, src->L, src->c0, src->cmax, src->cc, src->ccmax, src->act};
    rte_status st = mgnet_create(&cfg, stream, out);
    if (st != RTE_OK) return st;
    mgnet* n = *out;
    MG_GUARD_BEGIN
    check(cudaStreamSynchronize(src->stream), "sync");
    check(cudaMemcpyAsync(n->p, src->p, n->np * 4, cudaMemcpyDeviceToDevice, n->stream), "d2d");
    n->prec = src->prec;
    n->loss = src->loss;
    n->fault = src->fault;
    check(cudaStreamSynchronize(n->stream), "sync");
    ++n->version;
    return RTE_OK;
    MG_GUARD_END(n)
}

RTE_API void mgnet_destroy(mgnet* n) {
    if (!n) return;
    // the network's stream is the one of the context it ran with last, which
    // may be gone by now: wait for the whole device instead
    cudaDeviceSynchronize();
    for (auto& kv : n->feats)
        if (kv.second.block) cudaFree(kv.second.block);
    if (n->ws) cudaFree(n->ws);
    if (n->tc_ws) cudaFree(n->tc_ws);
    if (n->tcw) cudaFree(n->tcw);
    if (n->lscr) cudaFree(n->lscr);
    if (n->p) cudaFree(n->p);
    if (n->fin64) cudaFree(n->fin64);
    if (n->d_scal) cudaFree(n->d_scal);
    if (n->h_scal) cudaFreeHost(n->h_scal);
    delete n;
}

RTE_API int64_t mgnet_param_count(const mgnet* n) { return n ? (int64_t)n->np : -1; }

RTE_API rte_status mgnet_inject_fault(mgnet* n, int kind) {
    if (!n || (kind != MGNET_FAULT_NONE && kind != MGNET_FAULT_NAN)) {
        set_error(nullptr, "bad argument (MGNET_FAULT_NONE or MGNET_FAULT_NAN)");
        return RTE_EINVAL;
    }
    n->fault = kind;
    return RTE_OK;
}

RTE_API rte_status mgnet_get_config(const mgnet* n, mgnet_config* cfg) {
    if (!n || !cfg) { set_error(nullptr, "NULL argument"); return RTE_EINVAL; }
    *cfg = mgnet_config{n->M, n->L, n->c0, n->cmax, n->cc, n->ccmax, n->act};
    return RTE_OK;
}

RTE_API rte_status mgnet_set_precision(mgnet* n, int precision) {
    if (!n || (precision != MGNET_FP32 && precision != MGNET_BF16)) {
        set_error(nullptr, "bad argument (precision MGNET_FP32 or MGNET_BF16)");
        return RTE_EINVAL;
    }
    n->prec = precision;
    return RTE_OK;
}

RTE_API int mgnet_get_precision(const mgnet* n) { return n ? n->prec : -1; }

RTE_API rte_status mgnet_set_loss(mgnet* n, int kind) {
    if (!n || (kind != MGNET_LOSS_PLAIN && kind != MGNET_LOSS_FILTERED)) {
        set_error(nullptr, "bad argument (MGNET_LOSS_PLAIN or MGNET_LOSS_FILTERED)");
        return RTE_EINVAL;
    }
    n->loss = kind;
    return RTE_OK;
}

RTE_API int mgnet_get_loss(const mgnet* n) { return n ? n->loss : -1; }

RTE_API int mgnet_kernel_status(int reset) {
    try {
        return nn::conv_tc_status(reset != 0);
    } catch (...) {
        return -1;
    }
}

RTE_API rte_status mgnet_set_params(mgnet* n, const float* host, int64_t count) {
    if (!n || !host || count != (int64_t)n->np) { set_error(nullptr, "bad argument"); return RTE_EINVAL; }
    MG_GUARD_BEGIN
    check(cudaMemcpyAsync(n->p, host, n->np * 4, cudaMemcpyHostToDevice, n->stream), "h2d");
    check(cudaMemsetAsync(n->m, 0, n->np * 8, n->stream), "memset");
    check(cudaStreamSynchronize(n->stream), "sync");
    n->step = 0;
    ++n->version;
    return RTE_OK;
    MG_GUARD_END(n)
}

RTE_API rte_status mgnet_get_params(mgnet* n, float* host, int64_t count) {
    if (!n || !host || count != (int64_t)n->np) { set_error(nullptr, "bad argument"); return RTE_EINVAL; }
    MG_GUARD_BEGIN
    check(cudaMemcpyAsync(host, n->p, n->np * 4, cudaMemcpyDeviceToHost, n->stream), "d2h");
    check(cudaStreamSynchronize(n->stream), "sync");
    return RTE_OK;
    MG_GUARD_END(n)
}

RTE_API rte_status mgnet_precond(mgnet* n, rte_ctx* ctx, const double* r_dev, float* z_dev) {
    if (!n || !ctx || !r_dev || !z_dev) { set_error(nullptr, "NULL argument"); return RTE_EINVAL; }
    MG_GUARD_BEGIN
    mgnet_precondition(n, ctx, r_dev, z_dev);
    return RTE_OK;
    MG_GUARD_END(n)
}

RTE_API rte_status mgnet_apply(mgnet* n, rte_ctx* ctx, const double* r_dev, double* z_dev) {
    if (!n || !ctx || !r_dev || !z_dev) { set_error(nullptr, "NULL argument"); return RTE_EINVAL; }
    MG_GUARD_BEGIN
    Acts a = workspace(n, 2, ctx->I);
    mgnet_precondition(n, ctx, r_dev, a.gtmp);
    launch_block_apply(ctx, false, a.gtmp, false, z_dev, true);
    return RTE_OK;
    MG_GUARD_END(n)
}

static rte_status loss_grad_impl(mgnet* n, rte_ctx* ctx, const double* const* r_dev, int batch,
                                 double* loss_out) {
    if (!n || !ctx || !r_dev || batch < 1 || batch > 16) {
        set_error(nullptr, "bad argument (batch in [1, 16])");
        return RTE_EINVAL;
    }
    MG_GUARD_BEGIN
    check_ctx(n, ctx);
    for (int b = 0; b < batch; ++b)
        if (!r_dev[b]) throw StatusError{RTE_EINVAL, "NULL sample"};
    Features& F = features(n, ctx, true);
    const int Bw = batch < 2 ? 2 : batch;
    Acts a = workspace(n, Bw, ctx->I);
    load_inputs(n, ctx, r_dev, batch, a);
    forward(n, F, a, batch, ctx->I, true);
    const double loss = loss_and_seed(n, ctx, a, batch);
    check(cudaMemsetAsync(n->g, 0, n->np * 4, n->stream), "memset");
    backward(n, F, a, ctx, batch, ctx->I);
    if (loss_out) *loss_out = loss;
    return RTE_OK;
    MG_GUARD_END(n)
}

RTE_API rte_status mgnet_loss_grad(mgnet* n, rte_ctx* ctx, const double* const* r_dev, int batch,
                                   double* loss_out, float* grad_host) {
    rte_status st = loss_grad_impl(n, ctx, r_dev, batch, loss_out);
    if (st != RTE_OK || !grad_host) return st;
    MG_GUARD_BEGIN
    check(cudaMemcpyAsync(grad_host, n->g, n->np * 4, cudaMemcpyDeviceToHost, n->stream), "d2h");
    check(cudaStreamSynchronize(n->stream), "sync");
    return RTE_OK;
    MG_GUARD_END(n)
}

RTE_API rte_status mgnet_train_step(mgnet* n, rte_ctx* ctx, const double* const* r_dev, int batch,
                                    double lr, double* loss_out) {
    rte_status st = loss_grad_impl(n, ctx, r_dev, batch, loss_out);
    if (st != RTE_OK) return st;
    MG_GUARD_BEGIN
    ++n->step;
    nn::adam(n->p, n->g, n->m, n->v, n->np, (float)lr, n->step, n->stream);
    ++n->version;
    return RTE_OK;
    MG_GUARD_END(n)
}

// File format: "MGNET002", int32 M, levels, c0, cmax, cc, ccmax, act, int64 count,
// count float32 parameters, uint32 checksum (sum of the 32-bit words).
RTE_API rte_status mgnet_save(mgnet* n, const char* path) {
    if (!n || !path) { set_error(nullptr, "NULL argument"); return RTE_EINVAL; }
    MG_GUARD_BEGIN
    // weights, then the Adam moments m and v (p, g, m, v are consecutive)
    std::vector<float> h(3 * n->np);
    check(cudaMemcpyAsync(h.data(), n->p, n->np * 4, cudaMemcpyDeviceToHost, n->stream), "d2h");
    check(cudaMemcpyAsync(h.data() + n->np, n->m, 2 * n->np * 4, cudaMemcpyDeviceToHost, n->stream), "d2h");
    check(cudaStreamSynchronize(n->stream), "sync");
    FILE* f = std::fopen(path, "wb");
    if (!f) throw StatusError{RTE_EINVAL, "cannot open file for writing"};
    const int32_t hdr[7] = {n->M, n->L, n->c0, n->cmax, n->cc, n->ccmax, n->act};
    const int64_t cnt = (int64_t)n->np, step = n->step;
    uint32_t sum = (uint32_t)step;
    for (size_t i = 0; i < h.size(); ++i) { uint32_t w; std::memcpy(&w, &h[i], 4); sum += w; }
    bool ok = std::fwrite("MGNET003", 1, 8, f) == 8 && std::fwrite(hdr, 4, 7, f) == 7 &&
              std::fwrite(&cnt, 8, 1, f) == 1 && std::fwrite(&step, 8, 1, f) == 1 &&
              std::fwrite(h.data(), 4, h.size(), f) == h.size() && std::fwrite(&sum, 4, 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) throw StatusError{RTE_EINVAL, "write failed"};
    return RTE_OK;
    MG_GUARD_END(n)
}

RTE_API rte_status mgnet_load(mgnet* n, const char* path) {
    if (!n || !path) { set_error(nullptr, "NULL argument"); return RTE_EINVAL; }
    MG_GUARD_BEGIN
    FILE* f = std::fopen(path, "rb");
    if (!f) throw StatusError{RTE_EINVAL, "cannot open file"};
    char magic[8];
    int32_t hdr[7];
    int64_t cnt = 0, step = 0;
    bool ok = std::fread(magic, 1, 8, f) == 8;
    const bool v3 = ok && std::memcmp(magic, "MGNET003", 8) == 0;
    ok = ok && (v3 || std::memcmp(magic, "MGNET002", 8) == 0) && std::fread(hdr, 4, 7, f) == 7 &&
         std::fread(&cnt, 8, 1, f) == 1 && (!v3 || std::fread(&step, 8, 1, f) == 1);
    const int32_t want[7] = {n->M, n->L, n->c0, n->cmax, n->cc, n->ccmax, n->act};
    ok = ok && std::memcmp(hdr, want, sizeof(want)) == 0 && cnt == (int64_t)n->np && step >= 0;
    const size_t floats = ok ? (v3 ? 3 : 1) * n->np : 0;
    std::vector<float> h(floats);
    uint32_t sum = (uint32_t)step, stored = 0;
    ok = ok && std::fread(h.data(), 4, floats, f) == floats && std::fread(&stored, 4, 1, f) == 1;
    std::fclose(f);
    if (ok)
        for (size_t i = 0; i < floats; ++i) { uint32_t w; std::memcpy(&w, &h[i], 4); sum += w; }
    if (!ok || sum != stored) throw StatusError{RTE_EINVAL, "not a matching MGNET002/003 file or bad checksum"};
    const rte_status st = mgnet_set_params(n, h.data(), cnt);      // also resets the Adam state
    if (st != RTE_OK || !v3) return st;
    check(cudaMemcpyAsync(n->m, h.data() + n->np, 2 * n->np * 4, cudaMemcpyHostToDevice, n->stream), "h2d");
    check(cudaStreamSynchronize(n->stream), "sync");
    n->step = (int)step;
    return RTE_OK;
    MG_GUARD_END(n)
}

}  // extern "C"
