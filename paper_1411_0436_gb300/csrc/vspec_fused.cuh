// vspec_fused.cuh — one-pass fused channelizer for dual-pol, 2048..32768 channels.
//
// A thread-block cluster of K = N1/16 CTAs (one per SM) channelizes one
// spectrum at a time and loops over its share of the spectra, so the PFB
// delay line and the spectral accumulators stay on chip for the whole call
// and the int8 input is the only HBM traffic (§4 of arXiv 1411.0436:
// pre-filter, FFT, detect, accumulate).
//
// N = N1 * N2 with N2 = 128, n = n1 + N1 n2, k = k2 + N2 k1 (four-step):
//   * column phase — CTA j owns the 16 columns n1 in [16 j, 16 j + 16) and all
//     128 rows: pre-filter (§4, PFB) of its 2048 samples, then the 128-point
//     column DFTs over n2 in shared memory (in-place DIF passes; output
//     position pos holds k2 = digit-reversal of pos);
//   * exchange — after a cluster barrier, CTA j reads the R = 128/K rows
//     pos in [R j, R j + R) of every CTA's column tile through distributed
//     shared memory, multiplying by W_N^(n1 k2) on the way;
//   * row phase — the N1-point row DFTs over n1, whose last pass (radix 4) is
//     fused with detection (§4: X^2, Y^2, Re XY*, Im XY*) and accumulation
//     into registers owned by the same thread for every spectrum (§4,
//     accumulate).
// Column tiles are double-buffered, so one cluster barrier per spectrum is
// enough; the row DFTs of spectrum s-1 run between the barrier's arrive and
// wait of spectrum s. At the end every CTA writes its accumulators once to
// the cluster's slice of the partial-sum buffer; reduce_kernel adds the
// clusters and scatters to channel order.
#pragma once
#include <cooperative_groups.h>

#include "vspec_kernels.cuh"

namespace vspec {
namespace fused {

namespace cg = cooperative_groups;

constexpr int kThreads = 512;
constexpr int kN2 = 128;
constexpr int kCols = 16;  // columns per CTA: 64-byte rows of dual-pol int8

// Radix plans. Column DFT (length 128) and row DFT (length N1, last radix 4
// so each thread owns exactly four channels).
__host__ __device__ constexpr int col_radix(int i) { return i == 0 ? 8 : 4; }
constexpr int kColPasses = 3;  // 8 * 4 * 4 = 128

__host__ __device__ constexpr int row_passes(int logn1) {
    return logn1 == 8 ? 3 : logn1 == 7 ? 3 : logn1 == 6 ? 3 : 2;
}
__host__ __device__ constexpr int row_radix(int logn1, int i) {
    // 256 = 8*8*4, 128 = 8*4*4, 64 = 4*4*4, 32 = 8*4, 16 = 4*4
    return logn1 == 8 ? (i < 2 ? 8 : 4)
         : logn1 == 7 ? (i == 0 ? 8 : 4)
         : logn1 == 6 ? 4
         : logn1 == 5 ? (i == 0 ? 8 : 4)
         : 4;
}

struct Params {
    const int8_t *in;        // int8 [time][2][re, im]
    const float *coef;       // h[t * N + n], t < P
    const float2 *twA;       // column-pass twiddles (Pass::off layout)
    const float2 *twB;       // row-pass twiddles
    const float2 *twZ;       // [pos][n1] = W_N^(n1 k2(pos))
    float4 *partial;         // [cluster][pos][posB]
    int P;                   // taps (1 in direct mode)
    int nspectra;
    int nclusters;
    Pass colp[kColPasses];
    Pass rowp[3];
};

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

// ------------------------------------------------------------- passes ---

template <int R, int LB>
__device__ __forceinline__ void col_pass(float4 *cb, const float2 *tw) {
    constexpr int M = LB / R;
    constexpr int NB = kCols * (kN2 / R);
    for (int u = threadIdx.x; u < NB; u += kThreads) {
        const int c = u & (kCols - 1), bj = u / kCols;
        const int b = bj / M, j = bj % M;
        const int base = b * LB + j;
        float4 v[R];
#pragma unroll
        for (int q = 0; q < R; q++) v[q] = cb[(base + q * M) * kCols + c];
        Dft<R>::run(v);
        if constexpr (M > 1) {
            const float2 *t = tw + j * (R - 1);
#pragma unroll
            for (int q = 1; q < R; q++) v[q] = cmul(v[q], __ldg(t + q - 1));
        }
#pragma unroll
        for (int q = 0; q < R; q++) cb[(base + q * M) * kCols + c] = v[q];
    }
}

template <int LOGN1, int R, int LB>
__device__ __forceinline__ void row_pass(float4 *rb, const float2 *tw) {
    constexpr int N1 = 1 << LOGN1;
    constexpr int RS = N1 + N1 / 16;
    constexpr int ROWS = 2048 / N1;
    constexpr int M = LB / R;
    constexpr int PER_ROW = N1 / R;
    constexpr int NB = ROWS * PER_ROW;
    for (int u = threadIdx.x; u < NB; u += kThreads) {
        const int r = u / PER_ROW, w = u % PER_ROW;
        const int b = w / M, j = w % M;
        const int base = b * LB + j;
        float4 *row = rb + r * RS;
        float4 v[R];
#pragma unroll
        for (int q = 0; q < R; q++) v[q] = row[pad16(base + q * M)];
        Dft<R>::run(v);
        if constexpr (M > 1) {
            const float2 *t = tw + j * (R - 1);
#pragma unroll
            for (int q = 1; q < R; q++) v[q] = cmul(v[q], __ldg(t + q - 1));
        }
#pragma unroll
        for (int q = 0; q < R; q++) row[pad16(base + q * M)] = v[q];
    }
}

// Last row pass (radix 4, one butterfly per thread): DFT, detect, accumulate.
template <int LOGN1>
__device__ __forceinline__ void row_last_detect(const float4 *rb, float4 (&acc)[4]) {
    constexpr int N1 = 1 << LOGN1;
    constexpr int RS = N1 + N1 / 16;
    constexpr int PER_ROW = N1 / 4;
    const int u = threadIdx.x;
    const int r = u / PER_ROW, b = u % PER_ROW;
    const float4 *row = rb + r * RS;
    float4 v[4];
#pragma unroll
    for (int q = 0; q < 4; q++) v[q] = row[pad16(4 * b + q)];
    Dft<4>::run(v);
#pragma unroll
    for (int q = 0; q < 4; q++) acc_add<2>(acc[q], v[q]);
}

template <int LOGN1>
__device__ __forceinline__ void row_fft_detect(float4 *rb, const Params &p, float4 (&acc)[4]) {
    constexpr int N1 = 1 << LOGN1;
    constexpr int NP = row_passes(LOGN1);
    // all passes but the last, then the fused last pass
    if constexpr (NP == 3) {
        constexpr int R0 = row_radix(LOGN1, 0), R1 = row_radix(LOGN1, 1);
        row_pass<LOGN1, R0, N1>(rb, p.twB + p.rowp[0].off);
        __syncthreads();
        row_pass<LOGN1, R1, N1 / R0>(rb, p.twB + p.rowp[1].off);
        __syncthreads();
    } else {
        constexpr int R0 = row_radix(LOGN1, 0);
        row_pass<LOGN1, R0, N1>(rb, p.twB + p.rowp[0].off);
        __syncthreads();
    }
    row_last_detect<LOGN1>(rb, acc);
}

// --------------------------------------------------- tensor memory ---
// The PFB delay line lives in tensor memory (TMEM, 128 lanes x 512 columns of
// 32 bits per SM). Warp w may only touch lanes 32 (w % 4) .. +31, so the 16
// warps of the CTA split the columns four ways: thread (warp w, lane l) owns
// TMEM lane 32 (w % 4) + l, columns 128 (w / 4) .. +127, i.e. 8 frame slots of
// 16 floats (its 4 samples x re/im of both polarisations).

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(dst)), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};"
        :: "r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
           "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
           "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
           "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
           "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
           "r"(__float_as_uint(v[15]))
        : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// The 16 floats of one frame of this thread's 4 samples from four int8 words.
__device__ __forceinline__ void unpack4(const uint32_t (&w)[4], float (&v)[16]) {
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const uint32_t wx = w[i] ^ 0x80808080u;
#pragma unroll
        for (int k = 0; k < 4; k++) v[4 * i + k] = unpack_byte(wx, k);
    }
}

// ------------------------------------------------------------- kernel ---

// PT: taps (8 for the PFB, 1 for direct mode).
template <int LOGN1, int PT>
__global__ void __launch_bounds__(kThreads, 1) fused_kernel(const __grid_constant__ Params p) {
    constexpr int N1 = 1 << LOGN1;
    constexpr int N = N1 * kN2;
    constexpr int K = N1 / kCols;        // CTAs per cluster
    constexpr int R = kN2 / K;           // rows per CTA in the row phase
    constexpr int RS = N1 + N1 / 16;
    constexpr int TILE = kN2 * kCols;    // float4 per column tile (2048)

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *colbuf = reinterpret_cast<float4 *>(smem_raw);          // [2][128][16]
    float4 *rowbuf = colbuf + 2 * TILE;                              // [R][RS]
    float4 *coefs = rowbuf + R * RS;                                 // [PT][512]: 4 samples' h
    __shared__ uint32_t tmem_base_slot;

    cg::cluster_group cluster = cg::this_cluster();
    const int j = (int)cluster.block_rank();
    const int cl = blockIdx.x / K;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;

    const int s_beg = (int)((long long)p.nspectra * cl / p.nclusters);
    const int s_end = (int)((long long)p.nspectra * (cl + 1) / p.nclusters);

    // This thread's samples in the column phase: column c, rows n2 + 32 i.
    const int c = tid & (kCols - 1);
    const int n2b = tid >> 4;
    const long long n0 = (long long)j * kCols + c + (long long)N1 * n2b;  // first sample
    const unsigned int *in4 = reinterpret_cast<const unsigned int *>(p.in);  // one dual-pol sample
    auto load_frame = [&](long long f, uint32_t (&w)[4]) {
#pragma unroll
        for (int i = 0; i < 4; i++) w[i] = __ldg(in4 + f * N + n0 + (long long)N1 * 32 * i);
    };

#pragma unroll
    for (int t = 0; t < PT; t++) {
        float4 h;
        h.x = __ldg(p.coef + (size_t)t * N + n0);
        h.y = __ldg(p.coef + (size_t)t * N + n0 + N1 * 32);
        h.z = __ldg(p.coef + (size_t)t * N + n0 + N1 * 64);
        h.w = __ldg(p.coef + (size_t)t * N + n0 + N1 * 96);
        coefs[t * kThreads + tid] = h;
    }

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

    // W_N^(n1 k2) for the four elements this thread gathers each spectrum.
    float2 twg[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int e = tid + kThreads * i;
        const int r = e >> LOGN1, n1 = e & (N1 - 1);
        twg[i] = __ldg(p.twZ + (size_t)(R * j + r) * N1 + n1);
    }

    float4 acc[4];
#pragma unroll
    for (int q = 0; q < 4; q++) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);

    if (s_beg < s_end) {
        // delay line: frames s_beg .. s_beg + PT - 2 into their TMEM slots (frame f -> slot f % 8)
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
            const int buf = s & 1;
            float4 *cb = colbuf + buf * TILE;
            // ---- pre-filter (§4, PFB): y = sum_t h[t N + n] x[(s + t) N + n]
            float y[16];
            {
                float v[16];
                unpack4(nxt, v);  // newest frame s + PT - 1
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
                cb[(n2b + 32 * i) * kCols + c] = make_float4(y[4 * i], y[4 * i + 1], y[4 * i + 2], y[4 * i + 3]);
            __syncthreads();
            // ---- column DFTs over n2 (length 128)
            col_pass<col_radix(0), 128>(cb, p.twA + p.colp[0].off);
            __syncthreads();
            col_pass<col_radix(1), 128 / col_radix(0)>(cb, p.twA + p.colp[1].off);
            __syncthreads();
            col_pass<col_radix(2), 128 / (col_radix(0) * col_radix(1))>(cb, p.twA + p.colp[2].off);
            // ---- exchange: the barrier also publishes this CTA's tile
            cluster.barrier_arrive();
            if (s + 1 < s_end) load_frame((long long)s + PT, nxt);  // newest frame of s + 1
            if (s > s_beg) row_fft_detect<LOGN1>(rowbuf, p, acc);  // spectrum s - 1
            __syncthreads();
            cluster.barrier_wait();
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int e = tid + kThreads * i;
                const int r = e >> LOGN1, n1 = e & (N1 - 1);
                const float4 *src = cluster.map_shared_rank(cb, n1 / kCols);
                const float4 v = src[(R * j + r) * kCols + (n1 & (kCols - 1))];
                rowbuf[r * RS + pad16(n1)] = cmul(v, twg[i]);
            }
            __syncthreads();
        }
        row_fft_detect<LOGN1>(rowbuf, p, acc);  // last spectrum
    }
    // no CTA may leave while others can still read its tiles
    cluster.sync();

    if constexpr (PT > 1) {
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
        if (warp == 0) tmem_dealloc(tmem_base_slot, 512);
    }

    // accumulators -> this cluster's partial sums, [pos][posB]
    constexpr int PER_ROW = N1 / 4;
    const int r = tid / PER_ROW, b = tid % PER_ROW;
    float4 *dst = p.partial + (size_t)cl * N + (size_t)(R * j + r) * N1 + 4 * b;
#pragma unroll
    for (int q = 0; q < 4; q++) dst[q] = acc[q];
}

// Dynamic shared memory: two column tiles, the row tile and the coefficients.
// Always above half an SM's shared memory, so one CTA per SM (the kernel
// takes all 512 TMEM columns).
__host__ __device__ constexpr size_t smem_bytes(int logn1, int pt) {
    return (size_t)(2 * kN2 * kCols) * 16 + (size_t)(kN2 / ((1 << logn1) / kCols)) *
           ((1 << logn1) + (1 << logn1) / 16) * 16 + (size_t)(pt < 8 ? 8 : pt) * kThreads * 16;
}

}  // namespace fused
}  // namespace vspec
