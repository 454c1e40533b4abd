// Response apply o_C = R_C z_C on the tensor cores (tcgen05), for media whose
// per-cell blocks are interpolated in ln tau from tabulated nodes (Sec. 2.2:
// R_C = T_out,C G_C^{-1} depends on a cell only through its material and its
// optical thickness tau_C).
//
// With R_C = sum_p w_Cp R_p over the eight nodes p of the cell's stencil,
//     o_C = sum_q w_Cq (R_q z_C)
// over the nodes q of a tile of cells, w_Cq = 0 outside the cell's stencil.
// A tile is up to 128 consecutive cells of the cell list ordered by stencil,
// spanning at most kMaxTileNodes nodes.  Per node q the product
// U_q = Z R_q^T (Z: the tile's z vectors as rows) is one accumulation of
// M = 128 cells (TMEM lanes) x N = 2M outputs (TMEM columns) x K = 2M inputs;
// the epilogue warps add w_Cq U_q into registers while the MMAs of node q + 1
// run into the other accumulator buffer.  The dense contraction replaces the
// stream of the per-cell R_C from HBM (4 (2M)^2 bytes a cell) by (2M)^2 MMA
// work a cell and node, the node tables staying in L2.
//
// FP32 accuracy from BF16 operands: z and R_q are split into three BF16 parts
// each (an FP32 x = x0 + x1 + x2 exactly, |x1| <= 2^-8 |x0|, |x2| <= 2^-16
// |x0|), and the six products x_a y_b with a + b <= 2 are accumulated in FP32;
// the dropped ones are below 2^-24 of |x||y|.  The Lagrange weights enter the
// epilogue as float pairs (hi + lo), so that every cell's weights still sum to
// one: rounded to FP32 they would give each R_C a gain or loss of O(2^-24).
//
// Layout: the tiles read and write whole rows in the order of the cell list
// ([N][2M], row pos for cell cells[pos]); k_to_tiles and the gathers convert
// from and to the direction-major vectors with coalesced accesses on both
// sides.
//
// Roles (320 threads): warp 0 issues the bulk copies of the node tables into
// a ring of stages; warp 1 allocates tensor memory and one thread of it
// issues the MMAs; warps 2..9 build the tile's Z operand in shared memory
// and run the epilogue, two warps per TMEM lane quarter (warp w reads lanes
// 32 (w mod 4) ..), each with half of the outputs of its 32 cells.  Every
// wait is bounded: on expiry the CTA records it in g_resp_tc_status, drains
// its copies, writes NaN outputs, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "async_ptx.h"
#include "df64.h"
#include "rte_internal.h"

namespace rte {
namespace {

using namespace ::rte::ptx;

constexpr int kCells = 128;          // cells per tile = MMA M = TMEM lanes
constexpr int kParts = 3;            // BF16 parts of an FP32 value
constexpr int kKch = 32;             // inputs j per staged chunk of a node
constexpr int kStages = 4;
constexpr int kEpiWarps = 8;         // Z build and epilogue: two warps per TMEM lane quarter
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kMaxTileNodes = 16;    // nodes a tile may span

__device__ int g_resp_tc_status;     // 1 once a bounded wait expired

struct RespTcArgs {
    const float* zt;                 // [N][2M] the input in tile order (row pos = cell cells[pos])
    float* ot;                       // [N][2M] the output R z in tile order
    const int4* tiles;               // (first position, cells, first node, nodes)
    const int* first;                // [N] first stencil node at each position
    const float* w16;                // [N][16] Lagrange weights at each position: 8 hi, then 8 lo
    const uint16_t* nodes;           // node tables, BF16 parts (layout below)
};

// Byte offset of element (r, k) in a K-major no-swizzle operand of rows r and
// kdim K elements: 8-row x 16-byte core matrices, adjacent in K 128 bytes
// apart, adjacent in r (kdim / 8) * 128 bytes apart.
__host__ __device__ constexpr uint32_t kmajor_off(int r, int k, int kdim) {
    return (uint32_t)((r >> 3) * (kdim / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void split3(float x, uint32_t& h0, uint32_t& h1, uint32_t& h2) {
    const __nv_bfloat16 b0 = __float2bfloat16_rn(x);
    const float r1 = __fsub_rn(x, __bfloat162float(b0));        // exact
    const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
    const float r2 = __fsub_rn(r1, __bfloat162float(b1));       // exact
    const __nv_bfloat16 b2 = __float2bfloat16_rn(r2);
    h0 = __bfloat16_as_ushort(b0);
    h1 = __bfloat16_as_ushort(b1);
    h2 = __bfloat16_as_ushort(b2);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

// the MMA warp and the epilogue warps: Z is in shared memory
__device__ __forceinline__ void bar_sync_build() {
    asm volatile("bar.sync 1, %0;" ::"n"(32 + 32 * kEpiWarps) : "memory");
}

// Node tables: for node q and chunk c of kKch inputs, the three parts of
// R_q[i][c kKch + k] (i < NO, k < kKch) one after the other, each NO x kKch
// in the K-major layout: stage (q, c) is one contiguous block.
template <int NO>
__global__ void k_pack_nodes(int J, const double* __restrict__ Rn, uint16_t* __restrict__ out) {
    constexpr int NCH = NO / kKch;
    const int64_t total = (int64_t)J * NO * NO;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(e / (NO * NO));
        const int rem = (int)(e - (int64_t)q * NO * NO);
        const int j = rem / NO, i = rem - j * NO;               // Rn[q][j][i] = R_q[i][j]
        uint32_t h[3];
        split3((float)Rn[e], h[0], h[1], h[2]);
        const int c = j / kKch, k = j - c * kKch;
        uint16_t* blk = out + ((size_t)q * NCH + c) * kParts * NO * kKch;
        const uint32_t off = kmajor_off(i, k, kKch) / 2;
#pragma unroll
        for (int p = 0; p < kParts; ++p) blk[(size_t)p * NO * kKch + off] = (uint16_t)h[p];
    }
}

template <int NO>
__global__ void __launch_bounds__(kThreads, 1) k_response_tc(const __grid_constant__ RespTcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int NCH = NO / kKch;
    constexpr int HALF = NO / 2;                              // outputs per epilogue thread
    constexpr uint32_t A_PART = kCells * NO * 2;             // one BF16 part of Z
    constexpr uint32_t B_PART = NO * kKch * 2;               // one part of a node chunk
    constexpr uint32_t STAGE = kParts * B_PART;
    // two accumulator buffers, each a main (z0 R0) and a correction (the five
    // small products) accumulator: the tensor core's FP32 accumulation is not
    // rounded to nearest, and keeping the small products apart leaves the main
    // sum eight additions per node instead of 48 (no systematic gain or loss)
    constexpr uint32_t NCOLS = 4 * NO;
    constexpr uint32_t IDESC = idesc_bf16(kCells, NO);
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], accf[2], acce[2], done;
    __shared__ uint32_t tslot;
    __shared__ int fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int4 tile = a.tiles[blockIdx.x];
    const int pos0 = tile.x, count = tile.y, q0 = tile.z, nq = tile.w;
    const uint32_t abase = saddr(smem), bbase = abase + kParts * A_PART;

    if (warp == 1) tc_alloc(&tslot, NCOLS);
    if (tid == 0) {
        fail = 0;
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], kEpiWarps);
        }
        mbar_init(&done, 1);
        mbar_init_fence();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;

    // epilogue warps 2..9: cell m of the tile (TMEM lane, warp w reads lanes
    // 32 (w mod 4) ..) and half h of its outputs, kept in registers
    const int m = 32 * (warp & 3) + lane;
    const int h = (warp - 2) >> 2;
    const bool live = warp >= 2 && m < count;
    float acc[HALF];
#pragma unroll
    for (int i = 0; i < HALF; ++i) acc[i] = 0.f;

    if (warp == 0) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            const int total = nq * NCH;
            const unsigned char* src = reinterpret_cast<const unsigned char*>(a.nodes) + (size_t)q0 * NCH * STAGE;
            int it = 0;
            for (; it < total; ++it) {
                const int s = it % kStages;
                if (it >= kStages && !mbar_wait(&empty[s], ((it / kStages) - 1) & 1)) {
                    fail = 1;
                    break;
                }
                mbar_expect(&full[s], STAGE);
                bulk_load(bbase + s * STAGE, src + (size_t)it * STAGE, STAGE, &full[s]);
            }
            // every copy issued has landed before the CTA may leave
            for (int u = std::max(0, it - kStages); u < it; ++u)
                if (!mbar_wait(&full[u % kStages], (u / kStages) & 1)) fail = 1;
        }
    } else if (warp == 1) {
        // --------------------------------------------------------- MMA issue
        bar_sync_build();
        if (lane == 0) {
            tc_fence_after();
            bool ok = true;
            int it = 0;
            for (int g = 0; g < nq && ok; ++g) {
                const int b = g & 1;
                if (g >= 2 && !mbar_wait(&acce[b], ((g >> 1) - 1) & 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dmain = tmem + (uint32_t)(b * 2 * NO), dcorr = dmain + (uint32_t)NO;
                uint32_t acc_main = 0, acc_corr = 0;
                for (int c = 0; c < NCH; ++c, ++it) {
                    const int s = it % kStages;
                    if (!mbar_wait(&full[s], (it / kStages) & 1)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sb = bbase + s * STAGE;
#pragma unroll
                    for (int ks = 0; ks < kKch / 16; ++ks) {
                        const uint32_t aoff = (uint32_t)((c * kKch + ks * 16) / 8) * 128;
                        const uint32_t boff = (uint32_t)ks * 256;
                        // the six products z_pa R_pb, pa + pb <= 2
                        auto mma = [&](int pa, int pb, uint32_t d, uint32_t& accum) {
                            const uint64_t ad = sdesc(abase + pa * A_PART + aoff, 128, NO * 16);
                            const uint64_t bd = sdesc(sb + pb * B_PART + boff, 128, (kKch / 8) * 128);
                            tc_mma(d, ad, bd, IDESC, accum);
                            accum = 1;
                        };
                        mma(2, 0, dcorr, acc_corr);
                        mma(1, 1, dcorr, acc_corr);
                        mma(0, 2, dcorr, acc_corr);
                        mma(1, 0, dcorr, acc_corr);
                        mma(0, 1, dcorr, acc_corr);
                        mma(0, 0, dmain, acc_main);
                    }
                    tc_commit(&empty[s]);
                }
                if (!ok) break;
                tc_commit(&accf[b]);
            }
            tc_commit(&done);
            if (!mbar_wait(&done, 0)) ok = false;
            if (!ok) fail = 1;
        }
    } else {
        // ------------------------------------------- Z operand, then epilogue
        // this thread splits inputs j of half h of its cell's row of Z, a
        // contiguous row of the tile-ordered input
        constexpr int OCT = NO / 16;                          // octets of j per half
        constexpr int GRP = OCT < 4 ? OCT : 4;                // octets per round of loads
        const float4* zrow = reinterpret_cast<const float4*>(a.zt + (size_t)(pos0 + m) * NO);
        const uint32_t arow = abase + kmajor_off(m, 0, NO);
#pragma unroll 1
        for (int o0 = h * OCT; o0 < (h + 1) * OCT; o0 += GRP) {
            float4 v4[GRP * 2];
#pragma unroll
            for (int u = 0; u < GRP * 2; ++u) v4[u] = live ? __ldg(zrow + o0 * 2 + u) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int o8 = 0; o8 < GRP; ++o8) {
                const float v[8] = {v4[2 * o8].x, v4[2 * o8].y, v4[2 * o8].z, v4[2 * o8].w,
                                    v4[2 * o8 + 1].x, v4[2 * o8 + 1].y, v4[2 * o8 + 1].z, v4[2 * o8 + 1].w};
                uint32_t p[3][4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    uint32_t l0, l1, l2, h0, h1, h2;
                    split3(v[2 * e], l0, l1, l2);
                    split3(v[2 * e + 1], h0, h1, h2);
                    p[0][e] = l0 | (h0 << 16);
                    p[1][e] = l1 | (h1 << 16);
                    p[2][e] = l2 | (h2 << 16);
                }
                const uint32_t ad = arow + (uint32_t)(o0 + o8) * 128;
#pragma unroll
                for (int q = 0; q < 3; ++q) st_shared_v4(ad + q * A_PART, p[q][0], p[q][1], p[q][2], p[q][3]);
            }
        }
        fence_proxy_async();
        bar_sync_build();

        // the weights as float pairs (w = hi + lo to 2^-48): a cell's weights
        // sum to one, and an FP32 rounding of them would scale its whole R_C by
        // 1 + O(2^-24), a gain or loss comparable to the absorption of a
        // diffusive medium
        int f = -(1 << 30);
        float wh[8], wl[8];
#pragma unroll
        for (int p = 0; p < 8; ++p) wh[p] = wl[p] = 0.f;
        if (live) {
            f = __ldg(a.first + pos0 + m);
            const float4* wp = reinterpret_cast<const float4*>(a.w16 + (size_t)(pos0 + m) * 16);
            const float4 h0 = __ldg(wp), h1 = __ldg(wp + 1), l0 = __ldg(wp + 2), l1 = __ldg(wp + 3);
            wh[0] = h0.x; wh[1] = h0.y; wh[2] = h0.z; wh[3] = h0.w;
            wh[4] = h1.x; wh[5] = h1.y; wh[6] = h1.z; wh[7] = h1.w;
            wl[0] = l0.x; wl[1] = l0.y; wl[2] = l0.z; wl[3] = l0.w;
            wl[4] = l1.x; wl[5] = l1.y; wl[6] = l1.z; wl[7] = l1.w;
        }
        const uint32_t lanes = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(h * HALF);
        for (int g = 0; g < nq; ++g) {
            const int b = g & 1;
            // the warp leaves together: the loads below are warp-collective
            if (!__all_sync(0xffffffffu, mbar_wait(&accf[b], (g >> 1) & 1))) {
                fail = 1;
                break;
            }
            tc_fence_after();
            const int p = q0 + g - f;
            float wth = 0.f, wtl = 0.f;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                wth = (p == u) ? wh[u] : wth;
                wtl = (p == u) ? wl[u] : wtl;
            }
            if (__any_sync(0xffffffffu, wth != 0.f)) {
                const uint32_t tm = lanes + (uint32_t)(b * 2 * NO), tc = tm + (uint32_t)NO;
                if constexpr (HALF % 32 == 0) {
#pragma unroll
                    for (int c = 0; c < HALF; c += 32) {
                        float v[32], e[32];
                        tc_ld32(tm + (uint32_t)c, v);
                        tc_ld32(tc + (uint32_t)c, e);
#pragma unroll
                        for (int u = 0; u < 32; ++u) {
                            const float x = __fadd_rn(v[u], e[u]);
                            acc[c + u] = fmaf(wtl, x, fmaf(wth, x, acc[c + u]));
                        }
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < HALF; c += 16) {
                        float v[16], e[16];
                        tc_ld16(tm + (uint32_t)c, v);
                        tc_ld16(tc + (uint32_t)c, e);
#pragma unroll
                        for (int u = 0; u < 16; ++u) {
                            const float x = __fadd_rn(v[u], e[u]);
                            acc[c + u] = fmaf(wtl, x, fmaf(wth, x, acc[c + u]));
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[b]);
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (live) {
        // this cell's half row of the tile-ordered output
        const bool bad = fail != 0;
        float4* orow = reinterpret_cast<float4*>(a.ot + (size_t)(pos0 + m) * NO + h * HALF);
        const float nanv = __int_as_float(0x7fc00000);
#pragma unroll
        for (int i = 0; i < HALF / 4; ++i)
            orow[i] = bad ? make_float4(nanv, nanv, nanv, nanv)
                          : make_float4(acc[4 * i], acc[4 * i + 1], acc[4 * i + 2], acc[4 * i + 3]);
    }
    if (warp == 1) {
        __syncwarp();
        tc_dealloc(tmem, NCOLS);
    }
    if (tid == 0 && fail) atomicExch(&g_resp_tc_status, 1);
}

template <int NO>
constexpr size_t resp_tc_smem() {
    return (size_t)kParts * kCells * NO * 2 + (size_t)kStages * kParts * NO * kKch * 2;
}

template <int NO>
void launch_t(const RespTcArgs& args, int ntiles, cudaStream_t st) {
    auto kern = k_response_tc<NO>;
    raise_smem_limit((const void*)kern, resp_tc_smem<NO>());
    kern<<<ntiles, kThreads, resp_tc_smem<NO>(), st>>>(args);
    check(cudaGetLastError(), "k_response_tc");
}

// ------------------------------------------------------------ tile order
// The tiles take their cells' input rows and write their output rows in the
// order of the cell list (row pos = cell cells[pos], 2M contiguous floats),
// so that the tensor-core kernel moves whole rows; these kernels convert
// between that order and the direction-major vectors [2M][N] with both sides
// coalesced: a block of 32 consecutive cells is staged transposed in shared
// memory.

constexpr int kPermCells = 32;

// zt[pos_of[c]][j] = z[j N + c]
template <int NO, typename TIN>
__global__ void __launch_bounds__(256) k_to_tiles(int N, const TIN* __restrict__ z, const int* __restrict__ pos_of,
                                                  float* __restrict__ zt) {
    constexpr int PER = NO * kPermCells / 256;                 // elements per thread
    __shared__ float sb[kPermCells * (NO + 1)];
    const int c0 = blockIdx.x * kPermCells;
    float v[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {                            // all loads in flight, rows coalesced
        const int e = threadIdx.x + k * 256, j = e / kPermCells, c = c0 + e % kPermCells;
        v[k] = c < N ? (float)__ldg(z + (size_t)j * N + c) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int e = threadIdx.x + k * 256, j = e / kPermCells, cc = e % kPermCells;
        sb[cc * (NO + 1) + j] = v[k];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int cc = warp; cc < kPermCells; cc += 8) {            // one contiguous row per cell
        const int c = c0 + cc;
        if (c >= N) break;
        float* dst = zt + (size_t)__ldg(pos_of + c) * NO;
#pragma unroll
        for (int j = lane; j < NO; j += 32) dst[j] = sb[cc * (NO + 1) + j];
    }
}

// The neighbour value of row (f, j) of cell c (P o, o in tile order): the
// neighbour across face f returns its row (f ^ 1, j); zero on the boundary.
// Stages, for the block's 32 cells, every row of P o transposed in sb
// [2M][33] (the neighbours' face blocks of M/2 floats are read whole).
template <int NO>
__device__ __forceinline__ void stage_neighbour_rows(int I, int c0, const float* __restrict__ ot,
                                                     const int* __restrict__ pos_of, float* sb, int* npos) {
    constexpr int M2 = NO / 4, PER = NO * kPermCells / 256;
    const int N = I * I;
    if (threadIdx.x < 4 * kPermCells) {                        // the neighbours' positions
        const int f = threadIdx.x / kPermCells, c = c0 + threadIdx.x % kPermCells;
        int p = -1;
        if (c < N) {
            const int iy = c / I, ix = c - iy * I;
            int nb = -1;
            if (f == 0 && ix > 0) nb = c - 1;
            if (f == 1 && ix < I - 1) nb = c + 1;
            if (f == 2 && iy > 0) nb = c - I;
            if (f == 3 && iy < I - 1) nb = c + I;
            if (nb >= 0) p = __ldg(pos_of + nb);
        }
        npos[threadIdx.x] = p;
    }
    __syncthreads();
    float v[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {                            // all loads in flight
        const int e = threadIdx.x + k * 256;
        const int f = e / (kPermCells * M2), rem = e % (kPermCells * M2);
        const int cc = rem / M2, j = rem % M2;
        const int p = npos[f * kPermCells + cc];
        v[k] = p >= 0 ? __ldg(ot + (size_t)p * NO + (f ^ 1) * M2 + j) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int e = threadIdx.x + k * 256;
        const int f = e / (kPermCells * M2), rem = e % (kPermCells * M2);
        const int cc = rem / M2, j = rem % M2;
        sb[(f * M2 + j) * (kPermCells + 1) + cc] = v[k];
    }
    __syncthreads();
}

// df64 w = v - P o as gather_df_run, o in tile order
template <int NO>
__device__ void gather_tiles_df_run(int I, const float* __restrict__ vh, const float* __restrict__ vl,
                                    const float* __restrict__ ot, const int* __restrict__ pos_of,
                                    float* __restrict__ w, int bid, float* sb, int* npos) {
    constexpr int PER = NO * kPermCells / 256;
    const int N = I * I;
    const int64_t n = (int64_t)NO * N;
    const int c0 = bid * kPermCells;
    stage_neighbour_rows<NO>(I, c0, ot, pos_of, sb, npos);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int e = threadIdx.x + k * 256, row = e / kPermCells, cc = e % kPermCells, c = c0 + cc;
        if (c >= N) continue;
        const int64_t idx = (int64_t)row * N + c;
        const float ov = sb[row * (kPermCells + 1) + cc];
        float s, t, hh, ll;
        df::two_sum(vh[idx], -ov, s, t);
        if (vl) t = __fadd_rn(t, vl[idx]);
        df::two_sum(s, t, hh, ll);
        w[idx] = hh;
        w[n + idx] = ll;
    }
}

template <int NO>
__global__ void __launch_bounds__(256) k_gather_tiles_df(int I, const float* __restrict__ vh,
                                                         const float* __restrict__ vl,
                                                         const float* __restrict__ ot,
                                                         const int* __restrict__ pos_of, float* __restrict__ w) {
    __shared__ float sb[NO * (kPermCells + 1)];
    __shared__ int npos[4 * kPermCells];
    gather_tiles_df_run<NO>(I, vh, vl, ot, pos_of, w, blockIdx.x, sb, npos);
}

// w = v - P o as gather_run (the difference in FP64), o in tile order
template <int NO, typename TV, typename TW>
__global__ void __launch_bounds__(256) k_gather_tiles(int I, const TV* __restrict__ v,
                                                      const float* __restrict__ ot,
                                                      const int* __restrict__ pos_of, TW* __restrict__ w) {
    constexpr int PER = NO * kPermCells / 256;
    __shared__ float sb[NO * (kPermCells + 1)];
    __shared__ int npos[4 * kPermCells];
    const int N = I * I;
    const int c0 = blockIdx.x * kPermCells;
    stage_neighbour_rows<NO>(I, c0, ot, pos_of, sb, npos);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int e = threadIdx.x + k * 256, row = e / kPermCells, cc = e % kPermCells, c = c0 + cc;
        if (c >= N) continue;
        const int64_t idx = (int64_t)row * N + c;
        w[idx] = (TW)((double)v[idx] - (double)sb[row * (kPermCells + 1) + cc]);
    }
}

// grouped solves: the tile-ordered gathers of the items on the tensor-core path
__global__ void __launch_bounds__(256) k_gather_tiles_group(const GroupItem* __restrict__ items, int count) {
    __shared__ float sb[128 * (kPermCells + 1)];
    __shared__ int npos[4 * kPermCells];
    const GroupItem& it = items[group_item_of<&GroupItem::b_gt>(items, count)];
    const int bid = blockIdx.x - it.b_gt;
    if (it.M == 16) gather_tiles_df_run<32>(it.I, it.z, it.z_lo, it.o, it.pos_of, it.w, bid, sb, npos);
    if (it.M == 32) gather_tiles_df_run<64>(it.I, it.z, it.z_lo, it.o, it.pos_of, it.w, bid, sb, npos);
    if (it.M == 64) gather_tiles_df_run<128>(it.I, it.z, it.z_lo, it.o, it.pos_of, it.w, bid, sb, npos);
}

}  // namespace

bool response_tc_supported(int M) {
    const int NO = 2 * M;
    return NO == 32 || NO == 64 || NO == 128;
}

void build_response_tc(rte_ctx* ctx, const TabPlan& plan, const double* Rn) {
    const int M = ctx->M, NO = 2 * M, N = ctx->N;
    const int J = (int)plan.node_tau.size();
    if (!response_tc_supported(M) || J == 0) return;
    const cudaStream_t st = ctx->stream;
    // the first stencil node at each position, tiles of consecutive positions
    std::vector<int> first(N);
    for (const int4& b : plan.bins)
        for (int p = b.y; p < b.z; ++p) first[p] = b.x;
    std::vector<int4> tiles;
    for (int pos = 0; pos < N;) {
        const int q0 = first[pos];
        int end = pos;
        while (end < N && end - pos < kCells && first[end] + 8 - q0 <= kMaxTileNodes) ++end;
        tiles.push_back(make_int4(pos, end - pos, q0, first[end - 1] + 8 - q0));
        pos = end;
    }
    // the longest tiles start first
    std::stable_sort(tiles.begin(), tiles.end(), [](const int4& x, const int4& y) { return x.w > y.w; });
    double sum_nodes = 0.0;
    for (const int4& t : tiles) sum_nodes += t.w;

    ctx->tc_nodes = static_cast<uint16_t*>(dev_alloc(ctx, (size_t)J * kParts * NO * NO * sizeof(uint16_t)));
    ctx->tc_tiles = static_cast<int4*>(dev_alloc(ctx, tiles.size() * sizeof(int4)));
    ctx->tc_first = static_cast<int*>(dev_alloc(ctx, (size_t)N * sizeof(int)));
    ctx->tc_pos_of = static_cast<int*>(dev_alloc(ctx, (size_t)N * sizeof(int)));
    ctx->tc_w16 = ctx->tab_w16;              // Lagrange weights as float pairs
    auto up = [&](void* dst, const void* src, size_t bytes) {
        check(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st), "h2d (response tables)");
    };
    up(ctx->tc_tiles, tiles.data(), tiles.size() * sizeof(int4));
    std::vector<int> pos_of(N);
    for (int p = 0; p < N; ++p) pos_of[plan.cells[p]] = p;
    up(ctx->tc_pos_of, pos_of.data(), (size_t)N * sizeof(int));
    up(ctx->tc_first, first.data(), (size_t)N * sizeof(int));
    const int64_t total = (int64_t)J * NO * NO;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)ctx->num_sms * 16);
    if (NO == 32) k_pack_nodes<32><<<blocks, 256, 0, st>>>(J, Rn, ctx->tc_nodes);
    if (NO == 64) k_pack_nodes<64><<<blocks, 256, 0, st>>>(J, Rn, ctx->tc_nodes);
    if (NO == 128) k_pack_nodes<128><<<blocks, 256, 0, st>>>(J, Rn, ctx->tc_nodes);
    check(cudaGetLastError(), "k_pack_nodes");
    ctx->tc_ntiles = (int)tiles.size();
    ctx->tc_mma_flops = 6.0 * 2.0 * kCells * NO * NO * sum_nodes;
    // algorithmic device-memory bytes: z read, o written, the node tables once
    // (tiles re-read them from L2)
    ctx->tc_bytes = (double)ctx->n * 8 + (double)J * kParts * NO * NO * 2;
}

bool response_tc_active(const rte_ctx* ctx) {
    return ctx->tc_ntiles > 0 && ctx->response_path != RTE_RESPONSE_PER_CELL;
}

int tile_gather_blocks(const rte_ctx* ctx) { return (ctx->N + kPermCells - 1) / kPermCells; }

float* response_tc_output(rte_ctx* ctx) { return reinterpret_cast<float*>(ctx->trace_out); }

namespace {
// z (direction-major, float or double) -> the tile-ordered rows zt
template <int NO>
void to_tiles_t(rte_ctx* ctx, const void* z, bool z_is_double, float* zt, cudaStream_t st) {
    const int nb = tile_gather_blocks(ctx);
    if (z_is_double)
        k_to_tiles<NO, double><<<nb, 256, 0, st>>>(ctx->N, static_cast<const double*>(z), ctx->tc_pos_of, zt);
    else
        k_to_tiles<NO, float><<<nb, 256, 0, st>>>(ctx->N, static_cast<const float*>(z), ctx->tc_pos_of, zt);
    check(cudaGetLastError(), "k_to_tiles");
}

void to_tiles(rte_ctx* ctx, const void* z, bool z_is_double, cudaStream_t st) {
    float* zt = response_tc_output(ctx) + ctx->n;     // trace_out holds 2n doubles: room for both
    const int NO = 2 * ctx->M;
    if (NO == 32) to_tiles_t<32>(ctx, z, z_is_double, zt, st);
    if (NO == 64) to_tiles_t<64>(ctx, z, z_is_double, zt, st);
    if (NO == 128) to_tiles_t<128>(ctx, z, z_is_double, zt, st);
}

// the tiles' MMAs: zt -> ot (the tile-ordered output rows)
void tiles_mma(rte_ctx* ctx, cudaStream_t st) {
    const int NO = 2 * ctx->M;
    RespTcArgs args;
    args.ot = response_tc_output(ctx);
    args.zt = args.ot + ctx->n;
    args.tiles = ctx->tc_tiles;
    args.first = ctx->tc_first;
    args.w16 = ctx->tc_w16;
    args.nodes = ctx->tc_nodes;
    if (NO == 32) launch_t<32>(args, ctx->tc_ntiles, st);
    if (NO == 64) launch_t<64>(args, ctx->tc_ntiles, st);
    if (NO == 128) launch_t<128>(args, ctx->tc_ntiles, st);
}
}  // namespace

void launch_response_tc_on(rte_ctx* ctx, const void* z, bool z_is_double, cudaStream_t st) {
    to_tiles(ctx, z, z_is_double, st);
    tiles_mma(ctx, st);
}

void launch_response_tc(rte_ctx* ctx, const void* z, bool z_is_double) {
    {
        ProfScope ps(ctx, K_TILE_ORDER, (double)ctx->n * ((z_is_double ? 8 : 4) + 4) + (double)ctx->N * 4);
        to_tiles(ctx, z, z_is_double, ctx->stream);
    }
    ProfScope ps(ctx, K_RESPONSE_TC, ctx->tc_bytes, 1, ctx->tc_mma_flops);
    tiles_mma(ctx, ctx->stream);
}

void launch_gather_tiles_df(rte_ctx* ctx, const float* vh, const float* vl, float* w) {
    const int NO = 2 * ctx->M, nb = tile_gather_blocks(ctx);
    const float* ot = response_tc_output(ctx);
    ProfScope ps(ctx, K_GATHER, (double)ctx->n * ((vl ? 8 : 4) + 4 + 8) + (double)ctx->N * 4);
    if (NO == 32) k_gather_tiles_df<32><<<nb, 256, 0, ctx->stream>>>(ctx->I, vh, vl, ot, ctx->tc_pos_of, w);
    if (NO == 64) k_gather_tiles_df<64><<<nb, 256, 0, ctx->stream>>>(ctx->I, vh, vl, ot, ctx->tc_pos_of, w);
    if (NO == 128) k_gather_tiles_df<128><<<nb, 256, 0, ctx->stream>>>(ctx->I, vh, vl, ot, ctx->tc_pos_of, w);
    check(cudaGetLastError(), "k_gather_tiles_df");
}

namespace {
template <int NO>
void gather_tiles_t(rte_ctx* ctx, const void* v, bool v_is_double, void* w, bool w_is_double) {
    const int nb = tile_gather_blocks(ctx);
    const float* ot = response_tc_output(ctx);
    const int I = ctx->I;
    const int* pos = ctx->tc_pos_of;
    const cudaStream_t st = ctx->stream;
    if (v_is_double && w_is_double)
        k_gather_tiles<NO, double, double><<<nb, 256, 0, st>>>(I, (const double*)v, ot, pos, (double*)w);
    else if (!v_is_double && !w_is_double)
        k_gather_tiles<NO, float, float><<<nb, 256, 0, st>>>(I, (const float*)v, ot, pos, (float*)w);
    else if (!v_is_double && w_is_double)
        k_gather_tiles<NO, float, double><<<nb, 256, 0, st>>>(I, (const float*)v, ot, pos, (double*)w);
    else
        k_gather_tiles<NO, double, float><<<nb, 256, 0, st>>>(I, (const double*)v, ot, pos, (float*)w);
    check(cudaGetLastError(), "k_gather_tiles");
}
}  // namespace

void launch_gather_tiles(rte_ctx* ctx, const void* v, bool v_is_double, void* w, bool w_is_double) {
    ProfScope ps(ctx, K_GATHER, (double)ctx->n * ((v_is_double ? 8 : 4) + 4 + (w_is_double ? 8 : 4)));
    const int NO = 2 * ctx->M;
    if (NO == 32) gather_tiles_t<32>(ctx, v, v_is_double, w, w_is_double);
    if (NO == 64) gather_tiles_t<64>(ctx, v, v_is_double, w, w_is_double);
    if (NO == 128) gather_tiles_t<128>(ctx, v, v_is_double, w, w_is_double);
}

void launch_group_gather_tiles(const GroupItem* items_dev, int count, int blocks, cudaStream_t st) {
    if (blocks <= 0) return;
    k_gather_tiles_group<<<blocks, 256, 0, st>>>(items_dev, count);
    check(cudaGetLastError(), "k_gather_tiles_group");
}

int response_tc_timeout_flag(bool reset) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_resp_tc_status, sizeof(int)) != cudaSuccess) return -1;
    if (reset && v) {
        const int zero = 0;
        if (cudaMemcpyToSymbol(g_resp_tc_status, &zero, sizeof(int)) != cudaSuccess) return -1;
    }
    return v;
}

}  // namespace rte
