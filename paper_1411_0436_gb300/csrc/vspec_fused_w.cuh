// vspec_fused_w.cuh — one-pass fused channelizer for dual-pol, 32768 channels,
// with warp-local FFTs.
//
// Same decomposition as vspec_fused.cuh (a cluster of 16 CTAs per spectrum,
// N = 256 x 128, PFB delay line in tensor memory, accumulators in registers),
// but every DFT belongs to one warp, so a spectrum costs two CTA barriers:
//   * column phase — warp w owns column w of the CTA's 16 and runs its
//     128-point DFT (radix 4 in registers, radix 8 and radix 4 after two
//     warp-private exchanges through shared memory);
//   * row phase — warp 2r + p owns row r, polarisation p of the CTA's 8 rows
//     and runs its 256-point DFT (radix 8 in registers, radix 4 and radix 8
//     after two exchanges); the two warps of a row then meet at a 64-thread
//     named barrier and each detects (§4: X^2, Y^2, Re XY*, Im XY*) and
//     accumulates (§4) half of the row's channels.
#pragma once
#include <cooperative_groups.h>

#include "vspec_fused.cuh"
#include "vspec_kernels.cuh"

namespace vspec {
namespace fusedw {

namespace cg = cooperative_groups;
using fused::tmem_alloc;
using fused::tmem_dealloc;
using fused::tmem_fence_after;
using fused::tmem_fence_before;
using fused::tmem_ld16;
using fused::tmem_ld_wait;
using fused::tmem_relinquish;
using fused::tmem_st16;
using fused::tmem_st_wait;
using fused::unpack4;

constexpr int kThreads = 512;
constexpr int kN1 = 256, kN2 = 128, kN = kN1 * kN2;
constexpr int kK = 16;          // CTAs per cluster
constexpr int kR = 8;           // rows per CTA in the row phase
constexpr int kCols = 16;       // columns per CTA in the column phase
constexpr int kColStride = 129; // float4 per column (one pad element)
constexpr int kExpStride = 16;  // float4 per exported row (columns XOR-swizzled)
constexpr int kRowStride = 288; // float2 per (row, pol) unit: 256 + 256 / 8

// Radix plans (the plan builds its twiddle tables and digit-reversal maps
// from the same lists).
__host__ __device__ constexpr int col_radix(int i) { return i == 1 ? 8 : 4; }  // 4 * 8 * 4 = 128
__host__ __device__ constexpr int row_radix(int i) { return i == 1 ? 4 : 8; }  // 8 * 4 * 8 = 256
constexpr int kColTw0 = 0, kColTw1 = 32 * 3, kColTwN = 32 * 3 + 4 * 7;  // W_128^(jq), W_32^(jq)
constexpr int kRowTw0 = 0, kRowTw1 = 32 * 7, kRowTwN = 32 * 7 + 8 * 3;  // W_256^(jq), W_32^(jq)

struct Params {
    const int8_t *in;
    const float *coef;      // h[t * N + n]
    const float2 *twA;      // column-pass twiddles, kColTwN entries
    const float2 *twB;      // row-pass twiddles, kRowTwN entries
    const float2 *twZ;      // [pos][n1] = W_N^(n1 k2(pos))
    float4 *partial;        // [cluster][pos][posB]
    int nspectra;
    int nclusters;
};

__device__ __forceinline__ int rpad(int i) { return i + (i >> 3); }
// Column-tile swizzle: keeps the stride-1, stride-4 and radix-8 access patterns
// of the column DFT free of shared-memory bank conflicts.
__device__ __forceinline__ int colf(int i) { return i ^ ((i >> 3) & 7); }
// Exported row pos keeps column c at slot c ^ ((pos >> 2) & 7).
__device__ __forceinline__ int expf_slot(int pos, int c) { return pos * kExpStride + (c ^ ((pos >> 2) & 7)); }

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

__host__ __device__ constexpr size_t smem_bytes() {
    return (size_t)kCols * kColStride * 16 +        // column tile
           (size_t)2 * kN2 * kExpStride * 16 +      // exported rows, double-buffered
           (size_t)2 * kR * kRowStride * 8 +         // row units
           (size_t)8 * kThreads * 16 +               // coefficients
           (size_t)(kColTwN + kRowTwN) * 8;          // twiddles
}

// 128-point column DFT of column `c` (this warp), results exported by position.
__device__ __forceinline__ void column_dft(float4 *col, float4 *exp, const float2 *twc, int c, int lane) {
    // A1: radix 4 over n2 = lane + 32 i, twiddle W_128^(lane q)
    {
        float4 v[4];
#pragma unroll
        for (int i = 0; i < 4; i++) v[i] = col[colf(lane + 32 * i)];
        Dft<4>::run(v);
#pragma unroll
        for (int q = 1; q < 4; q++) v[q] = cmul(v[q], twc[kColTw0 + lane * 3 + q - 1]);
#pragma unroll
        for (int q = 0; q < 4; q++) col[colf(lane + 32 * q)] = v[q];
    }
    __syncwarp();
    // A2: radix 8 inside each 32-block, one polarisation per half-warp
    {
        float2 *col2 = reinterpret_cast<float2 *>(col);
        const int pol = lane >> 4, b = lane & 15, qb = b >> 2, j = b & 3;
        float2 v[8];
#pragma unroll
        for (int m = 0; m < 8; m++) v[m] = col2[colf(qb * 32 + j + 4 * m) * 2 + pol];
        Dft<8>::run(v);
#pragma unroll
        for (int m = 1; m < 8; m++) v[m] = cmul(v[m], twc[kColTw1 + j * 7 + m - 1]);
#pragma unroll
        for (int m = 0; m < 8; m++) col2[colf(qb * 32 + j + 4 * m) * 2 + pol] = v[m];
    }
    __syncwarp();
    // A3: radix 4 on contiguous blocks, export position 4 lane + q
    {
        float4 v[4];
#pragma unroll
        for (int q = 0; q < 4; q++) v[q] = col[colf(4 * lane + q)];
        Dft<4>::run(v);
#pragma unroll
        for (int q = 0; q < 4; q++) exp[expf_slot(4 * lane + q, c)] = v[q];
    }
}

// 256-point row DFT of one (row, pol) unit, in place, outputs by position.
__device__ __forceinline__ void row_dft(float2 *u, const float2 *twr, int lane) {
    {
        float2 v[8];
#pragma unroll
        for (int i = 0; i < 8; i++) v[i] = u[rpad(lane + 32 * i)];
        Dft<8>::run(v);
#pragma unroll
        for (int q = 1; q < 8; q++) v[q] = cmul(v[q], twr[kRowTw0 + lane * 7 + q - 1]);
#pragma unroll
        for (int q = 0; q < 8; q++) u[rpad(lane + 32 * q)] = v[q];
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int bu = lane + 32 * h, qb = bu >> 3, j = bu & 7;
        float2 v[4];
#pragma unroll
        for (int m = 0; m < 4; m++) v[m] = u[rpad(qb * 32 + j + 8 * m)];
        Dft<4>::run(v);
#pragma unroll
        for (int m = 1; m < 4; m++) v[m] = cmul(v[m], twr[kRowTw1 + j * 3 + m - 1]);
#pragma unroll
        for (int m = 0; m < 4; m++) u[rpad(qb * 32 + j + 8 * m)] = v[m];
    }
    __syncwarp();
    {
        float2 v[8];
#pragma unroll
        for (int q = 0; q < 8; q++) v[q] = u[rpad(8 * lane + q)];
        Dft<8>::run(v);
#pragma unroll
        for (int q = 0; q < 8; q++) u[rpad(8 * lane + q)] = v[q];
    }
}

__device__ __forceinline__ void named_barrier(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(nthreads) : "memory");
}

// Row DFTs of the CTA's 8 rows, then detection and accumulation.
__device__ __forceinline__ void rows_detect(float2 *rowbuf, const float2 *twr, int warp, int lane,
                                            float4 (&acc)[4]) {
    const int r = warp >> 1, p = warp & 1;
    row_dft(rowbuf + warp * kRowStride, twr, lane);
    named_barrier(1 + r, 64);
    const float2 *ux = rowbuf + (2 * r) * kRowStride, *uy = rowbuf + (2 * r + 1) * kRowStride;
#pragma unroll
    for (int qq = 0; qq < 4; qq++) {
        const int pos = 8 * lane + 4 * p + qq;
        const float2 x = ux[rpad(pos)], y = uy[rpad(pos)];
        acc_add<2>(acc[qq], make_float4(x.x, x.y, y.x, y.y));
    }
}

// PT: taps (8: PFB, 1: direct mode).
template <int PT>
__global__ void __launch_bounds__(kThreads, 1) fused_w_kernel(const __grid_constant__ Params p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *colbuf = reinterpret_cast<float4 *>(smem_raw);                      // [16][129]
    float4 *expbuf = colbuf + kCols * kColStride;                               // [2][128][17]
    float2 *rowbuf = reinterpret_cast<float2 *>(expbuf + 2 * kN2 * kExpStride); // [16][288]
    float4 *coefs = reinterpret_cast<float4 *>(rowbuf + 2 * kR * kRowStride);   // [8][512]
    float2 *twc = reinterpret_cast<float2 *>(coefs + 8 * kThreads);             // column twiddles
    float2 *twr = twc + kColTwN;                                                // row twiddles
    __shared__ uint32_t tmem_base_slot;

    cg::cluster_group cluster = cg::this_cluster();
    const int j = (int)cluster.block_rank();
    const int cl = blockIdx.x / kK;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const int s_beg = (int)((long long)p.nspectra * cl / p.nclusters);
    const int s_end = (int)((long long)p.nspectra * (cl + 1) / p.nclusters);

    // column-phase samples of this thread: column c, rows n2b + 32 i
    const int c = tid & (kCols - 1), n2b = tid >> 4;
    const long long n0 = (long long)j * kCols + c + (long long)kN1 * n2b;
    const unsigned int *in4 = reinterpret_cast<const unsigned int *>(p.in);
    auto load_frame = [&](long long f, uint32_t (&w)[4]) {
#pragma unroll
        for (int i = 0; i < 4; i++) w[i] = __ldg(in4 + f * kN + n0 + (long long)kN1 * 32 * i);
    };

#pragma unroll
    for (int t = 0; t < PT; t++) {
        float4 h;
        h.x = __ldg(p.coef + (size_t)t * kN + n0);
        h.y = __ldg(p.coef + (size_t)t * kN + n0 + kN1 * 32);
        h.z = __ldg(p.coef + (size_t)t * kN + n0 + kN1 * 64);
        h.w = __ldg(p.coef + (size_t)t * kN + n0 + kN1 * 96);
        coefs[t * kThreads + tid] = h;
    }
    for (int e = tid; e < kColTwN; e += kThreads) twc[e] = __ldg(p.twA + e);
    for (int e = tid; e < kRowTwN; e += kThreads) twr[e] = __ldg(p.twB + e);

    uint32_t taddr = 0;
    if constexpr (PT > 1) {
        if (warp == 0) {
            tmem_alloc(&tmem_base_slot, 512);
            tmem_relinquish();
        }
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
        taddr = tmem_base_slot + ((uint32_t)(32 * (warp & 3)) << 16) + 128u * (uint32_t)(warp >> 2);
    }

    float2 twg[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int e = tid + kThreads * i;
        twg[i] = __ldg(p.twZ + (size_t)(kR * j + (e >> 8)) * kN1 + (e & (kN1 - 1)));
    }
    float4 acc[4];
#pragma unroll
    for (int q = 0; q < 4; q++) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);

    if (s_beg < s_end) {
        if constexpr (PT > 1) {
            for (int t = 0; t < PT - 1; t++) {
                const long long f = s_beg + t;
                uint32_t w[4];
                load_frame(f, w);
                float v[16];
                unpack4(w, v);
                tmem_st16(taddr + 16u * (uint32_t)(f & 7), v);
            }
            tmem_st_wait();
        }
        uint32_t nxt[4];
        load_frame((long long)s_beg + PT - 1, nxt);
        __syncthreads();

        for (int s = s_beg; s < s_end; s++) {
            float4 *exp = expbuf + (s & 1) * kN2 * kExpStride;
            // ---- pre-filter (§4, PFB)
            float y[16];
            {
                float v[16];
                unpack4(nxt, v);
                const float4 h = coefs[(PT - 1) * kThreads + tid];
                const float hh[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
                for (int i = 0; i < 16; i++) y[i] = hh[i >> 2] * v[i];
                if constexpr (PT > 1) tmem_st16(taddr + 16u * (uint32_t)((s + PT - 1) & 7), v);
            }
            if constexpr (PT > 1) {
#pragma unroll
                for (int t = 0; t < PT - 1; t += 2) {
                    float a[16], b[16];
                    tmem_ld16(taddr + 16u * (uint32_t)((s + t) & 7), a);
                    if (t + 1 < PT - 1) tmem_ld16(taddr + 16u * (uint32_t)((s + t + 1) & 7), b);
                    tmem_ld_wait();
                    const float4 ha = coefs[t * kThreads + tid];
                    const float hha[4] = {ha.x, ha.y, ha.z, ha.w};
#pragma unroll
                    for (int i = 0; i < 16; i++) y[i] = fmaf(hha[i >> 2], a[i], y[i]);
                    if (t + 1 < PT - 1) {
                        const float4 hb = coefs[(t + 1) * kThreads + tid];
                        const float hhb[4] = {hb.x, hb.y, hb.z, hb.w};
#pragma unroll
                        for (int i = 0; i < 16; i++) y[i] = fmaf(hhb[i >> 2], b[i], y[i]);
                    }
                }
                tmem_st_wait();
            }
#pragma unroll
            for (int i = 0; i < 4; i++)
                colbuf[c * kColStride + colf(n2b + 32 * i)] = make_float4(y[4 * i], y[4 * i + 1], y[4 * i + 2], y[4 * i + 3]);
            __syncthreads();
            // ---- column DFT: warp w owns column w
            column_dft(colbuf + warp * kColStride, exp, twc, warp, lane);
            // ---- exchange: the cluster barrier publishes the exported rows
            cluster.barrier_arrive();
            if (s + 1 < s_end) load_frame((long long)s + PT, nxt);
            if (s > s_beg) rows_detect(rowbuf, twr, warp, lane, acc);  // spectrum s - 1
            __syncthreads();
            cluster.barrier_wait();
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int e = tid + kThreads * i;
                const int r = e >> 8, n1 = e & (kN1 - 1);
                const float4 *src = cluster.map_shared_rank(exp, n1 >> 4);
                const float4 v = cmul(src[expf_slot(kR * j + r, n1 & 15)], twg[i]);
                rowbuf[(2 * r) * kRowStride + rpad(n1)] = lo2(v);
                rowbuf[(2 * r + 1) * kRowStride + rpad(n1)] = hi2(v);
            }
        }
        __syncthreads();
        rows_detect(rowbuf, twr, warp, lane, acc);  // last spectrum
    }
    cluster.sync();

    if constexpr (PT > 1) {
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
        if (warp == 0) tmem_dealloc(tmem_base_slot, 512);
    }

    // accumulators -> partial[cl][pos][posB], pos = 8 j + r, posB = 8 lane + 4 p + qq
    const int r = warp >> 1, pp = warp & 1;
    float4 *dst = p.partial + (size_t)cl * kN + (size_t)(kR * j + r) * kN1 + 8 * lane + 4 * pp;
#pragma unroll
    for (int q = 0; q < 4; q++) dst[q] = acc[q];
}

}  // namespace fusedw
}  // namespace vspec
