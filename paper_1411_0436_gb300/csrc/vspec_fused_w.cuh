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
constexpr int kRowStride = 256; // float2 per (row, pol) unit (index-swizzled)

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

// Swizzle of a row unit (256 float2): bits 4, 5, 6 of the index flip bits
// 0..3 by 1, 10 and 4, keeping the gather, the three row passes and the
// fused detection free of shared-memory bank conflicts.
__device__ __forceinline__ int rpad(int i) {
    return i ^ (((i >> 4) & 1) * 1) ^ (((i >> 5) & 1) * 10) ^ (((i >> 6) & 1) * 4);
}
// Swizzle of a column plane (128 float2 of one polarisation): bits 4, 5, 6 of
// the index flip bits 0..3 by 1, 6 and 8, which keeps the three access
// patterns of the column DFT (stride 1, the radix-8 pattern, stride 4) free
// of shared-memory bank conflicts.
__device__ __forceinline__ int cswz(int i) {
    return i ^ (((i >> 4) & 1) * 1) ^ (((i >> 5) & 1) * 6) ^ (((i >> 6) & 1) * 8);
}
// int8 staging tile (one frame of the CTA's 128 x 16 samples, one 32-bit word
// per dual-pol sample): row n2 keeps column c at word c ^ ((n2 >> 1) & 15), so
// both the coalesced row-wise writes and the column-wise reads are free of
// bank conflicts.
__device__ __forceinline__ int rawslot(int n2, int c) { return n2 * 16 + (c ^ ((n2 >> 1) & 15)); }
// Exported row pos keeps column c at slot c ^ ((pos >> 2) & 7).
__device__ __forceinline__ int expf_slot(int pos, int c) { return pos * kExpStride + (c ^ ((pos >> 2) & 7)); }

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

__host__ __device__ constexpr size_t smem_bytes() {
    return (size_t)kN2 * kCols * 4 +                // int8 staging tile
           (size_t)2 * kCols * kN2 * 8 +            // column planes
           (size_t)2 * kN2 * kExpStride * 16 +      // exported rows, double-buffered
           (size_t)2 * kR * kRowStride * 8 +         // row units
           (size_t)8 * kThreads * 16 +               // coefficients
           (size_t)(kColTwN + kRowTwN) * 8;          // twiddles
}

// 128-point column DFT of column `c` (this warp) from its pre-filtered rows
// lane + 32 i held in registers; results exported by position.
__device__ __forceinline__ void column_dft(float4 (&v)[4], float2 *px, float2 *py, float4 *exp,
                                           const float2 (&tw1)[3], const float2 *twc, int c, int lane) {
    // A1: radix 4 over n2 = lane + 32 i, twiddle W_128^(lane q)
    Dft<4>::run(v);
#pragma unroll
    for (int q = 1; q < 4; q++) v[q] = cmul(v[q], tw1[q - 1]);
#pragma unroll
    for (int q = 0; q < 4; q++) {
        px[cswz(lane + 32 * q)] = make_float2(v[q].x, v[q].y);
        py[cswz(lane + 32 * q)] = make_float2(v[q].z, v[q].w);
    }
    __syncwarp();
    // A2: radix 8 inside each 32-block, one polarisation per half-warp
    {
        float2 *pl = (lane >> 4) ? py : px;
        const int b = lane & 15, qb = b >> 2, j = b & 3;
        float2 w[8];
#pragma unroll
        for (int m = 0; m < 8; m++) w[m] = pl[cswz(qb * 32 + j + 4 * m)];
        Dft<8>::run(w);
#pragma unroll
        for (int m = 1; m < 8; m++) w[m] = cmul(w[m], twc[kColTw1 + j * 7 + m - 1]);
#pragma unroll
        for (int m = 0; m < 8; m++) pl[cswz(qb * 32 + j + 4 * m)] = w[m];
    }
    __syncwarp();
    // A3: radix 4 on contiguous blocks, export position 4 lane + q
    {
        float4 u[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const float2 a = px[cswz(4 * lane + q)], b = py[cswz(4 * lane + q)];
            u[q] = make_float4(a.x, a.y, b.x, b.y);
        }
        Dft<4>::run(u);
#pragma unroll
        for (int q = 0; q < 4; q++) exp[expf_slot(4 * lane + q, c)] = u[q];
    }
}

__device__ __forceinline__ void named_barrier(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(nthreads) : "memory");
}

// Row DFTs of the CTA's 8 rows (warp 2 r + p: row r, polarisation p), fused
// with detection and accumulation. The first two passes run on the warp's own
// unit; the last radix-8 pass takes blocks 16 p .. 16 p + 15 of row r for
// both polarisations (lanes 0-15: X, lanes 16-31: Y), so after one shuffle
// each lane holds X and Y for four channels.
__device__ __forceinline__ void rows_detect(float2 *rowbuf, const float2 *twr, const float2 (&tw2)[3],
                                            int warp, int lane, float4 (&acc)[4]) {
    const int r = warp >> 1, p = warp & 1;
    float2 *u = rowbuf + warp * kRowStride;
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
        for (int m = 1; m < 4; m++) v[m] = cmul(v[m], tw2[m - 1]);  // W_32^(j m), j = lane & 7
#pragma unroll
        for (int m = 0; m < 4; m++) u[rpad(qb * 32 + j + 8 * m)] = v[m];
    }
    named_barrier(1 + r, 64);
    const int half = lane >> 4, b = 16 * p + (lane & 15);
    const float2 *src = rowbuf + (2 * r + half) * kRowStride;
    float2 v[8];
#pragma unroll
    for (int q = 0; q < 8; q++) v[q] = src[rpad(8 * b + q)];
    Dft<8>::run(v);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const float2 send = half ? v[k] : v[4 + k];
        float2 recv;
        recv.x = __shfl_xor_sync(0xffffffffu, send.x, 16);
        recv.y = __shfl_xor_sync(0xffffffffu, send.y, 16);
        const float2 x = half ? recv : v[k];
        const float2 y = half ? v[4 + k] : recv;
        acc_add<2>(acc[k], make_float4(x.x, x.y, y.x, y.y));
    }
}

// PT: taps (8: PFB, 1: direct mode).
template <int PT>
__global__ void __launch_bounds__(kThreads, 1) fused_w_kernel(const __grid_constant__ Params p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *raw = reinterpret_cast<uint32_t *>(smem_raw);                     // [128][16] words
    float2 *planes = reinterpret_cast<float2 *>(raw + kN2 * kCols);             // [2 pol][16][128]
    float4 *expbuf = reinterpret_cast<float4 *>(planes + 2 * kCols * kN2);      // [2][128][16]
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

    // Loading set (coalesced): column cl, rows n2b + 32 i. Compute set (the
    // pre-filter, its delay line and the column DFT): column `warp`, rows
    // lane + 32 i.
    const int cl_ = tid & (kCols - 1), n2b = tid >> 4;
    const long long n0 = (long long)j * kCols + cl_ + (long long)kN1 * n2b;
    const long long m0 = (long long)j * kCols + warp + (long long)kN1 * lane;
    const unsigned int *in4 = reinterpret_cast<const unsigned int *>(p.in);
    auto load_frame = [&](long long f, uint32_t (&w)[4]) {
#pragma unroll
        for (int i = 0; i < 4; i++) w[i] = __ldg(in4 + f * kN + n0 + (long long)kN1 * 32 * i);
    };
    auto stage = [&](const uint32_t (&w)[4]) {
#pragma unroll
        for (int i = 0; i < 4; i++) raw[rawslot(n2b + 32 * i, cl_)] = w[i];
    };
    auto unstage = [&](uint32_t (&w)[4]) {
#pragma unroll
        for (int i = 0; i < 4; i++) w[i] = raw[rawslot(lane + 32 * i, warp)];
    };

#pragma unroll
    for (int t = 0; t < PT; t++) {
        float4 h;
        h.x = __ldg(p.coef + (size_t)t * kN + m0);
        h.y = __ldg(p.coef + (size_t)t * kN + m0 + kN1 * 32);
        h.z = __ldg(p.coef + (size_t)t * kN + m0 + kN1 * 64);
        h.w = __ldg(p.coef + (size_t)t * kN + m0 + kN1 * 96);
        coefs[t * kThreads + tid] = h;
    }
    float2 tw1[3], tw2[3];
#pragma unroll
    for (int q = 1; q < 4; q++) {
        tw1[q - 1] = __ldg(p.twA + kColTw0 + lane * 3 + q - 1);
        tw2[q - 1] = __ldg(p.twB + kRowTw1 + (lane & 7) * 3 + q - 1);
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
        __syncthreads();
        if constexpr (PT > 1) {
            for (int t = 0; t < PT - 1; t++) {
                const long long f = s_beg + t;
                uint32_t w[4];
                load_frame(f, w);
                stage(w);
                __syncthreads();
                unstage(w);
                __syncthreads();
                float v[16];
                unpack4(w, v);
                tmem_st16(taddr + 16u * (uint32_t)(f & 7), v);
            }
            tmem_st_wait();
        }
        uint32_t nxt[4];
        load_frame((long long)s_beg + PT - 1, nxt);

        for (int s = s_beg; s < s_end; s++) {
            float4 *exp = expbuf + (s & 1) * kN2 * kExpStride;
            stage(nxt);
            __syncthreads();
            // ---- pre-filter (§4, PFB) of the compute set
            float y[16];
            {
                uint32_t w[4];
                unstage(w);
                float v[16];
                unpack4(w, v);
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
            // ---- column DFT: warp w owns column w
            {
                float4 v4[4];
#pragma unroll
                for (int i = 0; i < 4; i++) v4[i] = make_float4(y[4 * i], y[4 * i + 1], y[4 * i + 2], y[4 * i + 3]);
                column_dft(v4, planes + warp * kN2, planes + (kCols + warp) * kN2, exp, tw1, twc, warp, lane);
            }
            // ---- exchange: the cluster barrier publishes the exported rows
            cluster.barrier_arrive();
            if (s + 1 < s_end) load_frame((long long)s + PT, nxt);
            if (s > s_beg) rows_detect(rowbuf, twr, tw2, warp, lane, acc);  // spectrum s - 1
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
        rows_detect(rowbuf, twr, tw2, warp, lane, acc);  // last spectrum
    }
    cluster.sync();

    if constexpr (PT > 1) {
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
        if (warp == 0) tmem_dealloc(tmem_base_slot, 512);
    }

    // accumulators -> partial[cl][pos][posB], pos = 8 j + r,
    // posB = 8 (16 pp + lane % 16) + 4 (lane / 16) + k
    const int r = warp >> 1, pp = warp & 1;
    float4 *dst = p.partial + (size_t)cl * kN + (size_t)(kR * j + r) * kN1 +
                  8 * (16 * pp + (lane & 15)) + 4 * (lane >> 4);
#pragma unroll
    for (int q = 0; q < 4; q++) dst[q] = acc[q];
}

}  // namespace fusedw
}  // namespace vspec
