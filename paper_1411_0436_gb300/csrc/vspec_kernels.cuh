// vspec_kernels.cuh — device code of the channelizer (§4 of arXiv 1411.0436).
//
// The N-point DFT of every spectrum is split as N = N1 * N2 (four-step):
//   n = n1 + N1*n2,  k = k2 + N2*k1,
//   X[k2 + N2 k1] = sum_n1 W_N1^(n1 k1) [ W_N^(n1 k2) sum_n2 y[n1 + N1 n2] W_N2^(n2 k2) ].
// Kernel A (fir_colfft, or its register-column forms fir_colreg and
// fir_coldir) owns a tile of C consecutive columns n1 and all N2 rows across
// a run of spectra. Each thread keeps the last P frames of its samples in
// registers as fp32, so every input byte is read from memory once per run.
// It applies the pre-filter (§4, PFB), runs the column DFTs over n2 (in
// registers, or in passes through shared memory), multiplies by
// W_N^(n1 k2) and writes the chunk scratch Z. Kernel B (row2048 or the
// general rowfft_detect) owns rows k2 and runs the row DFTs over n1, fused
// with detection (§4: X^2, Y^2, Re XY*, Im XY*) and accumulation in
// registers or shared memory (§4, accumulate). A last small kernel adds the
// per-CTA partial sums into the caller's accumulator in channel order.
//
// Both kernels use in-place decimation-in-frequency passes: a pass of radix r
// over blocks of length lb reads v[q] = x[j + q*m] (m = lb / r), computes the
// r-point DFT, multiplies output q by W_lb^(j*q) and writes it back to
// x[j + q*m]. After all passes, position sum_i q_i * M_i holds output index
// q_1 + r_1 (q_2 + r_2 (q_3 + ...)); the plan precomputes those
// digit-reversal maps and only the final scatter into channel order uses them.
#pragma once
#include <cstdint>
#include <type_traits>
#include <utility>

#include "vspec_radix.cuh"

namespace vspec {

constexpr int kMaxPasses = 6;

// Bounds checks of the debug build (compiled with -DVSPEC_DEBUG): a failed
// check sets its bit in g_debug_flags and the guarded access is skipped;
// nothing traps. In the release build dbg_ok is `true` and costs nothing.
//   bit 0: chunk-scratch index (spectrum, row position, column) out of range
//   bit 1: input frame past the call's input
//   bit 2: partial-sum slot or position out of range
//   bit 3: tile index out of range
enum : unsigned { kDbgScratch = 1u, kDbgInput = 2u, kDbgSlot = 4u, kDbgTile = 8u };
#ifdef VSPEC_DEBUG
#ifdef VSPEC_NO_PLAN_TABLES
static __device__ unsigned int g_debug_flags;  // this translation unit's own word
#else
__device__ unsigned int g_debug_flags;
#endif
__device__ __forceinline__ bool dbg_ok(bool cond, unsigned bit) {
    if (!cond) atomicOr(&g_debug_flags, bit);
    return cond;
}
#else
__device__ __forceinline__ constexpr bool dbg_ok(bool, unsigned) { return true; }
#endif

template <int NPOL> struct Elem;
template <> struct Elem<1> {
    using T = float2;     // one complex sample
    using Acc = float;    // XX
};
template <> struct Elem<2> {
    using T = P2;         // both polarisations of one sample or channel, packed
    using Acc = float4;   // XX, YY, Re XY*, Im XY*
};

struct ColParams {
    const int8_t *in;    // sample m of pol p at in[(m * npol + p) * 2 + {0: re, 1: im}]
    const float *coef;   // pre-filter coefficients h[t * N + n], t < P (fp32)
    const float2 *twA;   // per-pass twiddles of the length-N2 column DFTs
    const float2 *twZ;   // [pos][n1]: W_N^(n1 * k2(pos)) (rows in pass-output order)
    void *Z;             // chunk scratch [s_local][pos][n1] of Elem::T
    int N, N1, N2, C, P, npass;
    int lC, lN2;         // log2 C, log2 N2
    Pass pass[kMaxPasses];
    long long s0;        // absolute index of the chunk's first spectrum
    int sc;              // spectra in this chunk
    int tiles;           // column tiles, N1 / C
    int G;               // tiles per group (tile_split); 0 or 1: no groups
    int win;             // direct mode with a window: multiply by coef (register-column kernels)
    // tensor-core column kernel only
    const unsigned char *dftop;  // the column DFT operand: fp16 hi part, then lo part (then, for
                                 // fir_coltc_kernel, the four-step twiddles times 2^-12)
    int *status;                 // set to 1 if a bounded wait for the tensor cores gave up
    unsigned wait_limit;         // polls of that wait
    int bterms;                  // fp16 parts of the fused tensor-core operand: 1 (hi) or 2 (hi, lo)
    long long nframes;           // frames the call's input holds (bounds checks of debug builds)
    // sub-band input read in place (register-column kernels): sample m of band
    // b is word m nsub + b of the input, [time][sub][pol]; nsub = 1: plain.
    // band = -1: every band in one launch, tile X being tile X / nsub of band
    // X mod nsub, band b's spectra at Z + b N with a spectrum stride of zstride
    int nsub = 1, band = 0;
    long long zstride = 0;  // scratch elements per spectrum (0: N)
};

struct RowParams {
    const void *Z;       // chunk scratch written by kernel A
    void *partial;       // [group][pos][posB] of Elem::Acc, accumulated into
    void *partial_comp;  // Kahan compensation of `partial` (compensated plans only)
    const float2 *twB;   // per-pass twiddles of the length-N1 row DFTs
    int N, N1, N2, RB, npass;
    int lN1, lRB;        // log2 N1, log2 RB
    Pass pass[kMaxPasses];
    int sc;              // spectra in this chunk
    int tiles;           // row tiles, N2 / RB
    int slots;           // partial-sum slots (span_slot bound)
    // N2 == 1 (the row is the whole transform): the first pass reads the
    // int8 input and applies the FIR itself instead of reading Z
    const int8_t *in;
    const float *coef;
    int P;
    long long s0;        // absolute index of the chunk's first spectrum
    int store;           // 1: every slot has exactly one writer this call, which stores (no zeroing)
    long long nframes;   // frames the call's input holds (bounds checks of debug builds)
};

// ------------------------------------------------------------ work split --
// A launch's work is tiles x sc (tile, spectrum) items, tile-major. Block k
// of n takes items [k T / n, (k+1) T / n), T = tiles * sc: equal shares to
// within one item, whatever the tile count, so one wave of CTAs is busy to
// the end. A block's items form at most a few runs of consecutive spectra of
// one tile (segments).
struct Span {
    long long lo, hi;
};
__device__ __forceinline__ Span block_span(int tiles, int sc) {
    const long long T = (long long)tiles * sc;
    return {T * blockIdx.x / gridDim.x, T * (blockIdx.x + 1) / gridDim.x};
}
// Rank of this block among the blocks whose items meet tile x: the first
// such block is the one holding item x * sc, the largest k with
// floor(k T / n) <= x * sc. Ranks are below n / tiles + 2.
__device__ __forceinline__ int span_slot(int tiles, int sc, int x) {
    const long long T = (long long)tiles * sc;
    const long long k_lo = (((long long)x * sc + 1) * gridDim.x - 1) / T;
    return (int)(blockIdx.x - k_lo);
}

// Kernel A's split: blocks come in groups of G consecutive blocks that take
// the same items of the tiles / G super-tiles (block_span over the groups),
// member r the r-th tile of each super-tile. G adjacent tiles share the
// input's 128-byte lines (a tile row is C samples), and a group reads them
// at about the same time, so each line comes from HBM once. Needs G | tiles
// and G | gridDim.x. Tile of super-tile item f: (f / sc) * G + r.
struct TileSplit {
    long long lo, hi;
    int G, r;
};
__device__ __forceinline__ TileSplit tile_split(int tiles, int sc, int G) {
    if (G < 1) G = 1;
    const int ng = gridDim.x / G, g = blockIdx.x / G;
    if (g >= ng) return {0, 0, G, 0};  // blocks past the last whole group: no items
    const long long T = (long long)(tiles / G) * sc;
    return {T * g / ng, T * (g + 1) / ng, G, (int)(blockIdx.x % G)};
}

// ---------------------------------------------------------------- unpack ---
// Exact int8 -> fp32: placing (b ^ 0x80) in the low mantissa byte of 2^23
// gives the float 2^23 + b + 128; subtracting 2^23 + 128 leaves b exactly.
__device__ __forceinline__ float unpack_byte(uint32_t wx, int i) {
    return __int_as_float(__byte_perm(wx, 0x4B000000u, 0x7540u + i)) - 8388736.0f;
}

// Both polarisations of one dual-pol input word (already ^ 0x80808080) as
// P2: the real parts are bytes 0 and 2, the imaginary parts bytes 1 and 3.
// The bias is removed with one paired add per part; exact as above.
__device__ __forceinline__ P2 unpack_p2(uint32_t wx) {
    const float2 bias = make_float2(-8388736.0f, -8388736.0f);
    const float2 r = make_float2(__int_as_float(__byte_perm(wx, 0x4B000000u, 0x7540u)),
                                 __int_as_float(__byte_perm(wx, 0x4B000000u, 0x7542u)));
    const float2 i = make_float2(__int_as_float(__byte_perm(wx, 0x4B000000u, 0x7541u)),
                                 __int_as_float(__byte_perm(wx, 0x4B000000u, 0x7543u)));
    return P2{__fadd2_rn(r, bias), __fadd2_rn(i, bias)};
}

// Global loads that do not allocate in L1 (data read once, such as the
// chunk scratch, so that it does not push reused tables out of L1).
__device__ __forceinline__ float4 ld_no_l1(const float4 *ptr) {
    float4 v;
    asm volatile("ld.global.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(ptr));
    return v;
}
__device__ __forceinline__ float2 ld_no_l1(const float2 *ptr) {
    float2 v;
    asm volatile("ld.global.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(ptr));
    return v;
}
__device__ __forceinline__ P2 ld_no_l1(const P2 *ptr) {
    const float4 e = ld_no_l1(reinterpret_cast<const float4 *>(ptr));
    return P2{make_float2(e.x, e.y), make_float2(e.z, e.w)};
}

template <int NPOL> __device__ __forceinline__ uint32_t load_raw(const int8_t *in, long long m);
template <> __device__ __forceinline__ uint32_t load_raw<2>(const int8_t *in, long long m) {
    return __ldg(reinterpret_cast<const unsigned int *>(in) + m);
}
template <> __device__ __forceinline__ uint32_t load_raw<1>(const int8_t *in, long long m) {
    return (uint32_t)__ldg(reinterpret_cast<const unsigned short *>(in) + m);
}

// ------------------------------------------------------ kernel A helpers ---

template <int R, int NPOL>
__device__ __forceinline__ void col_butterfly(const ColParams &p, typename Elem<NPOL>::T *data,
                                              typename Elem<NPOL>::T *Zs, const Pass ps,
                                              bool last, int c, int b, int j, int n1, const float2 *tws) {
    using T = typename Elem<NPOL>::T;
    const int C = p.C;
    const int base = b * ps.lb + j;
    T v[R];
#pragma unroll
    for (int q = 0; q < R; q++) v[q] = data[(base + q * ps.m) * C + c];
    Dft<R>::run(v);
    if (!last) {
        if (ps.m > 1) {
            const float2 *tw = p.twA + ps.off + j * (R - 1);
#pragma unroll
            for (int q = 1; q < R; q++) v[q] = cmul(v[q], __ldg(tw + q - 1));
        }
#pragma unroll
        for (int q = 0; q < R; q++) data[(base + q * ps.m) * C + c] = v[q];
    } else {
        // last pass: m == 1, outputs at positions base + q
#pragma unroll
        for (int q = 0; q < R; q++) {
            const size_t zi = (size_t)(base + q) * p.N1 + n1;
            if (dbg_ok(base + q < p.N2 && n1 < p.N1, kDbgScratch)) Zs[zi] = cmul(v[q], tws[(base + q) * C + c]);
        }
    }
}

// Column DFTs of a batch of nb spectra (data holds their pre-filter outputs,
// [spectrum][n2][c]), then W_N^(n1 k2) and the store into the chunk scratch.
// tws: the tile's four-step twiddles W_N^(n1 k2(pos)), [pos][c], in shared memory.
template <int NPOL, int RMAX>
__device__ __forceinline__ void col_fft_store(const ColParams &p, typename Elem<NPOL>::T *data,
                                              int x, int s_local0, int nb, const float2 *tws) {
    using T = typename Elem<NPOL>::T;
    const int C = p.C, N2 = p.N2;
    const int pts = N2 * C;
    const int n1_0 = x * C;
    if (p.npass == 0) {  // N2 == 1: the pre-filter output is the row itself
        for (int u = threadIdx.x; u < nb * C; u += blockDim.x) {
            const int sb = u >> p.lC, c = u & (C - 1);
            T *Zs = reinterpret_cast<T *>(p.Z) + (size_t)(s_local0 + sb) * p.N;
            Zs[n1_0 + c] = data[u];
        }
    }
    for (int ip = 0; ip < p.npass; ip++) {
        const Pass ps = p.pass[ip];
        const bool last = ip == p.npass - 1;
        const int lper = p.lC + p.lN2 - ps.lr;  // log2 of the butterflies per spectrum
        for (int u = threadIdx.x; u < (nb << lper); u += blockDim.x) {
            const int sb = u >> lper, w = u & ((1 << lper) - 1);
            const int c = w & (C - 1), bj = w >> p.lC;
            const int b = bj >> ps.lm, j = bj & (ps.m - 1);
            T *d = data + sb * pts;
            T *Zs = reinterpret_cast<T *>(p.Z) + (size_t)(s_local0 + sb) * p.N;
            if (ps.r == 2) col_butterfly<2, NPOL>(p, d, Zs, ps, last, c, b, j, n1_0 + c, tws);
            else if (ps.r == 4 || RMAX < 8) col_butterfly<4, NPOL>(p, d, Zs, ps, last, c, b, j, n1_0 + c, tws);
            else if (ps.r == 8 || RMAX < 16) col_butterfly<(RMAX < 8 ? 4 : 8), NPOL>(p, d, Zs, ps, last, c, b, j, n1_0 + c, tws);
            else col_butterfly<RMAX, NPOL>(p, d, Zs, ps, last, c, b, j, n1_0 + c, tws);
        }
        __syncthreads();
    }
    if (p.npass == 0) __syncthreads();
}

// Stage column tile x's four-step twiddles twZ[pos][x*C + c] into shared
// memory as [pos][c] (read once per run of spectra instead of per spectrum).
__device__ __forceinline__ void stage_tile_twiddles(const ColParams &p, float2 *tws, int x) {
    if (p.npass == 0) return;  // N2 == 1: no four-step twiddles
    const int pts = p.N2 * p.C;
    for (int e = threadIdx.x; e < pts; e += blockDim.x) {
        const int pos = e >> p.lC, c = e & (p.C - 1);
        tws[e] = __ldg(p.twZ + (size_t)pos * p.N1 + x * p.C + c);
    }
}

// f(std::integral_constant<int, U>) for every U of the sequence, or for the
// U below n.
template <typename F, int... U>
__device__ __forceinline__ void for_slots(F &&f, std::integer_sequence<int, U...>) {
    (f(std::integral_constant<int, U>{}), ...);
}
template <typename F, int... U>
__device__ __forceinline__ void for_slots_below(F &&f, int n, std::integer_sequence<int, U...>) {
    ((U < n ? f(std::integral_constant<int, U>{}) : void()), ...);
}

// Widest column butterfly kernel A may use next to its register window.
// Window registers per thread are ppt * pt * (2 npol + 1); an r-point
// butterfly holds r * 2 npol more floats.
__host__ __device__ constexpr int col_radix_cap(int npol, int pt, int ppt) {
    return ppt * pt * (2 * npol + 1) + 16 * 2 * npol <= 72 ? 16
         : ppt * pt * (2 * npol + 1) + 8 * 2 * npol <= 72 ? 8 : 4;
}

// ---------------------------------------------------------------- kernel A --
// PT: taps held in the register window (P rounded up; the leading PT - P taps
// have zero coefficients and read a clamped frame). PPT: samples per thread.
// Spectra are processed in batches of PT: the window rotates once per batch,
// so every slot index is a compile-time constant, and the batch's column
// DFTs then run together. The window stays live through the column DFTs, so
// the widest butterfly is capped by the window's register footprint; the
// plan builds its pass list with the same cap (col_radix_cap).
// One segment: spectra [s_beg, s_end) of the chunk for column tile x.
template <int NPOL, int PT, int PPT>
__device__ __forceinline__ void fir_colfft_segment(const ColParams &p, typename Elem<NPOL>::T *data, int x,
                                                   int s_beg, int s_end, const float2 *tws) {
    using T = typename Elem<NPOL>::T;
    constexpr int NC = 2 * NPOL;  // floats per sample
    const int C = p.C;
    const int pts = p.N2 * C;
    const int n1_0 = x * C;
    const int D = PT - p.P;  // leading zero taps

    // dual-pol with few window registers: the FIR runs on paired FP32
    // instructions (coefficients duplicated into register pairs)
    constexpr bool kPacked = NPOL == 2 && PPT * PT <= 8;
    long long n_pt[PPT];
    int sm_pt[PPT];
    float cf[PPT][PT];
    float2 cf2[kPacked ? PPT : 1][kPacked ? PT : 1];
#pragma unroll
    for (int i = 0; i < PPT; i++) {
        const int idx = threadIdx.x + i * blockDim.x;  // = n2 * C + c
        const int c = idx & (C - 1), n2 = idx >> p.lC;
        n_pt[i] = n1_0 + c + (long long)p.N1 * n2;
        sm_pt[i] = idx;
#pragma unroll
        for (int t = 0; t < PT; t++) {
            cf[i][t] = (t >= D) ? __ldg(p.coef + (size_t)(t - D) * p.N + n_pt[i]) : 0.0f;
            if constexpr (kPacked) cf2[i][t] = dup2(cf[i][t]);
        }
    }

    // Slot (s - s_beg + t) % PT of the window holds frame s + t - D.
    float win[kPacked ? 1 : PPT][kPacked ? 1 : PT][NC];
    P2 win2[kPacked ? PPT : 1][kPacked ? PT : 1];
    const long long sabs = p.s0 + s_beg;
#pragma unroll
    for (int t = 0; t < PT - 1; t++) {
        long long f = sabs - D + t;
        if (f < 0) f = 0;
#pragma unroll
        for (int i = 0; i < PPT; i++) {
            const uint32_t wx = dbg_ok(f < p.nframes, kDbgInput) ? load_raw<NPOL>(p.in, f * p.N + n_pt[i]) ^ 0x80808080u
                                                               : 0x80808080u;
            if constexpr (kPacked) {
                win2[i][t] = unpack_p2(wx);
            } else {
#pragma unroll
                for (int k = 0; k < NC; k++) win[i][t][k] = unpack_byte(wx, k);
            }
        }
    }

    // each batch's PT new frames are copied into shared memory with
    // asynchronous copies one batch ahead (double-buffered), so the FIR reads
    // them without waiting on HBM
    constexpr bool kStaged = true;
    constexpr int B = 2 * NPOL;  // bytes per sample
    unsigned char *raw = reinterpret_cast<unsigned char *>(const_cast<float2 *>(tws) + pts);  // [2][PT][pts]
    auto stage = [&](int sb, int buf) {
        const int nbb = min(PT, s_end - sb);
        // 16-byte chunks: per_row = C * B / 16 per tile row, N2 rows per frame
        const int lrow = p.lC + (NPOL == 2 ? 2 : 1) - 4, lframe = lrow + p.lN2;
        for (int e = threadIdx.x; e < (nbb << lframe); e += blockDim.x) {
            const int u = e >> lframe, r = e & ((1 << lframe) - 1);
            const int n2 = r >> lrow, ch = r & ((1 << lrow) - 1);
            const long long fr = p.s0 + sb + u + p.P - 1;  // newest frame of spectrum sb + u
            const unsigned char *src = reinterpret_cast<const unsigned char *>(p.in) +
                                       (fr * p.N + n1_0 + (long long)p.N1 * n2) * B + ch * 16;
            unsigned char *dst = raw + ((size_t)(buf * PT + u) * pts + n2 * C) * B + ch * 16;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                         :: "r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if constexpr (kStaged) stage(s_beg, 0);

    for (int s_base = s_beg, buf = 0; s_base < s_end; s_base += PT, buf ^= 1) {
        const int nb = min(PT, s_end - s_base);
        if constexpr (kStaged) {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncthreads();  // this batch's frames are visible; the other buffer is free
            if (s_base + PT < s_end) stage(s_base + PT, buf ^ 1);
        }
        // the FIR of one spectrum of the batch (slot u of the window rotation)
        auto fir_one = [&](auto uc) {
            constexpr int u = decltype(uc)::value;
            constexpr int snew = (u + PT - 1) % PT;
#pragma unroll
            for (int i = 0; i < PPT; i++) {
                uint32_t wx;
                if constexpr (kStaged) {
                    const unsigned char *rs = raw + ((size_t)(buf * PT + u) * pts + sm_pt[i]) * B;
                    if constexpr (NPOL == 2) wx = *reinterpret_cast<const uint32_t *>(rs);
                    else wx = *reinterpret_cast<const unsigned short *>(rs);
                } else {  // newest frame of spectrum s_base + u
                    wx = load_raw<NPOL>(p.in, (p.s0 + s_base + u + p.P - 1) * p.N + n_pt[i]);
                }
                wx ^= 0x80808080u;
                T *d = data + u * pts + sm_pt[i];
                if constexpr (kPacked) {
                    win2[i][snew] = unpack_p2(wx);
                    const P2 &w0 = win2[i][u % PT];
                    P2 y{__fmul2_rn(cf2[i][0], w0.re), __fmul2_rn(cf2[i][0], w0.im)};
#pragma unroll
                    for (int t = 1; t < PT; t++) {
                        const P2 &wt = win2[i][(u + t) % PT];
                        y.re = __ffma2_rn(cf2[i][t], wt.re, y.re);
                        y.im = __ffma2_rn(cf2[i][t], wt.im, y.im);
                    }
                    *d = y;
                } else {
#pragma unroll
                    for (int k = 0; k < NC; k++) win[i][snew][k] = unpack_byte(wx, k);
                    float y[NC];
#pragma unroll
                    for (int k = 0; k < NC; k++) y[k] = cf[i][0] * win[i][u % PT][k];
#pragma unroll
                    for (int t = 1; t < PT; t++) {
#pragma unroll
                        for (int k = 0; k < NC; k++) y[k] = fmaf(cf[i][t], win[i][(u + t) % PT][k], y[k]);
                    }
                    if constexpr (NPOL == 2) *d = make_p2(y[0], y[1], y[2], y[3]);
                    else *d = make_float2(y[0], y[1]);
                }
            }
        };
        // a full batch has no per-spectrum guards, so the PT spectra's
        // independent FMA chains interleave freely
        if (nb == PT) for_slots(fir_one, std::make_integer_sequence<int, PT>{});
        else for_slots_below(fir_one, nb, std::make_integer_sequence<int, PT>{});
        __syncthreads();
        col_fft_store<NPOL, col_radix_cap(NPOL, PT, PPT)>(p, data, x, s_base, nb, tws);
    }
}

template <int NPOL, int PT, int PPT>
__global__ void __launch_bounds__(512) fir_colfft_kernel(const __grid_constant__ ColParams p) {
    using T = typename Elem<NPOL>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *data = reinterpret_cast<T *>(smem_raw);  // [PT][N2][C]
    float2 *tws = reinterpret_cast<float2 *>(data + PT * p.N2 * p.C);  // [N2][C], then (PFB) raw frames
    const TileSplit sp = tile_split(p.tiles, p.sc, p.G);
    for (long long f = sp.lo; f < sp.hi;) {
        const long long base = f / p.sc * p.sc;  // first item of this super-tile
        const int x = (int)(f / p.sc) * sp.G + sp.r;
        const int s_end = (int)(min(sp.hi, base + p.sc) - base);
        // the barrier after the first batch's FIR orders the twiddle tile's
        // stores before their use; col_fft_store ends on a barrier, so the
        // next segment may overwrite data and the tile
        stage_tile_twiddles(p, tws, x);
        fir_colfft_segment<NPOL, PT, PPT>(p, data, x, (int)(f - base), s_end, tws);
        f = base + s_end;
    }
}

// Kernel A, register-column form: dual-pol PFB of at most 8 taps in tiles of
// 512 points (one per thread) with columns of N2 = 2 .. 128 points (nchan
// 2^12 .. 2^18 with 2048-point rows, 2^19 with 4096-point rows). The FIR
// stage is the same register
// window as above. Columns of at most 16 points (R1 == N2) are then whole
// length-N2 DFTs in registers, one column per thread, in natural output
// order (the plan's column pass list is the single radix-N2 pass, so
// pos = k2). Longer columns take two DIF passes, radix R1 = 8 then N2 / 8,
// the plan's pass list {8, N2/8}, with every index a compile-time function of
// the thread: the first pass's twiddles come from a small table in shared
// memory, the second pass writes the chunk scratch. Every output is
// multiplied by W_N^(n1 k2) on its way out. SPB spectra share a column
// stage, so that the 512 threads have whole butterflies to work on.
template <int N2, int R1 = N2>
struct ColReg {
    static constexpr int PT = 8, PTS = 512, C = PTS / N2;
    static constexpr bool kOnePass = R1 == N2;
    static constexpr int R2 = N2 / R1;  // second-pass radix (two-pass form)
    // spectra per column stage: enough that each pass has a butterfly per thread
    static constexpr int SPB = kOnePass ? (N2 > PT ? N2 : PT)
                                        : (PTS / (C * (R1 < R2 ? R1 : R2)) > PT ? PTS / (C * (R1 < R2 ? R1 : R2)) : PT);
    static constexpr int CPT = SPB * C / PTS;             // columns per thread (one pass)
    static constexpr int B1 = SPB * C * (N2 / R1) / PTS;  // first-pass butterflies per thread
    static constexpr int B2 = SPB * C * R1 / PTS;         // second-pass butterflies per thread
    static constexpr int TWC = kOnePass ? 0 : (N2 / R1) * (R1 - 1);  // first-pass twiddles
    // Narrow tiles (C < 8 in the two-pass form): an 8-lane phase of the second
    // pass spans 8 / C blocks b, C * R2 elements apart; C pad elements after
    // every C * R2 put them in different banks. Element i of a spectrum is at
    // pad(i); a spectrum takes SS elements.
    static constexpr int PADG = !kOnePass && C < 8 ? C * R2 : 0, PADW = C;
    static constexpr int SS = PTS + (PADG ? PTS / PADG * PADW : 0);
    __device__ static constexpr int pad(int i) { return PADG ? i + i / PADG * PADW : i; }
    // The twiddle tile likewise: a 16-lane phase of the second pass reads
    // 16 / C blocks b, R2 rows apart; C pad entries after every R2 rows.
    static constexpr int TWPAD = !kOnePass && C < 16 ? C : 0;
    static constexpr int TWS = PTS + (TWPAD ? R1 * TWPAD : 0);
    __device__ static constexpr int twi(int pos, int c) { return pos * C + c + (TWPAD ? pos / R2 * TWPAD : 0); }
    // data [SPB][SS] P2, twiddle tile [N2][C] float2 (TWS entries), raw frames
    // [2][SPB][PTS] u32, coefficients [PT][PTS] float, first-pass twiddles [TWC] float2
    static constexpr size_t smem = (size_t)SPB * SS * 16 + (size_t)TWS * 8 + 2 * (size_t)SPB * PTS * 4 +
                                   (size_t)PT * PTS * 4 + (size_t)TWC * 8;
    static_assert(smem <= 232448, "shared memory of one CTA");
    static_assert(kOnePass ? N2 <= 16 : (R1 == 8 && (N2 == 32 || N2 == 64 || N2 == 128)), "column shapes of this kernel");
    static_assert(B1 * PTS == SPB * C * (N2 / R1) && B2 * PTS == SPB * C * R1, "whole butterflies per thread");
};

// Tile x of the register-column kernel A over spectra s_beg .. s_end - 1 of
// a chunk: spectrum s of the chunk is absolute spectrum s0 + s and goes to
// Zc[s] (the chunk holds sc spectra). All PTS threads of the CTA take part;
// the function ends with a barrier. twc: load the first-pass twiddles (they
// stay in shared memory for later tiles of the same launch).
template <int N2, int R1>
__device__ __forceinline__ void colreg_tile(const ColParams &p, void *Zc, long long s0, int sc, int x, int s_beg,
                                            int s_end, unsigned char *smem_raw, bool load_twc, int band = 0) {
    using G = ColReg<N2, R1>;
    constexpr int PT = G::PT, PTS = G::PTS, C = G::C, SPB = G::SPB;
    constexpr int SS = G::SS;
    P2 *data = reinterpret_cast<P2 *>(smem_raw);                       // [SPB][SS]
    float2 *tws = reinterpret_cast<float2 *>(data + SPB * SS);         // [N2][C], at twi(pos, c)
    uint32_t *raw = reinterpret_cast<uint32_t *>(tws + G::TWS);        // [2][SPB][PTS]
    float *cfs = reinterpret_cast<float *>(raw + 2 * SPB * PTS);       // [PT][PTS]
    float2 *twc = reinterpret_cast<float2 *>(cfs + PT * PTS);          // [N2/R1][R1-1]
    const int t = threadIdx.x;                                         // point n2 * C + c
    const int D = PT - p.P;                                            // leading zero taps
    const size_t zs = p.zstride > 0 ? (size_t)p.zstride : (size_t)p.N;  // scratch spectrum stride
    // first-pass twiddles W_N2^(j q) (ordered before use by the loop's barriers)
    if (load_twc)
        for (int e = t; e < G::TWC; e += PTS) twc[e] = __ldg(p.twA + p.pass[0].off + e);
    {
        const int n1_0 = x * C;
        for (int e = t; e < PTS; e += PTS)  // W_N^(n1 k2), k2 = pos
            tws[G::twi(e / C, e % C)] = __ldg(p.twZ + (size_t)(e / C) * p.N1 + n1_0 + (e % C));

        const long long n_pt = n1_0 + (t % C) + (long long)p.N1 * (t / C);
        // the tile's coefficients, read back for every batch so that their
        // registers are free during the column DFTs (each thread reads only
        // what it wrote: no barrier needed)
#pragma unroll
        for (int k = 0; k < PT; k++) cfs[k * PTS + t] = k >= D ? __ldg(p.coef + (size_t)(k - D) * p.N + n_pt) : 0.f;
        // slot (s - s_beg + k) % PT of the window holds frame s + k - D
        P2 win[PT];
        const long long sabs = s0 + s_beg;
#pragma unroll
        for (int k = 0; k < PT - 1; k++) {
            long long fr = sabs - D + k;
            if (fr < 0) fr = 0;
            win[k] = unpack_p2((dbg_ok(fr < p.nframes, kDbgInput) ? load_raw<2>(p.in, (fr * p.N + n_pt) * p.nsub + band)
                                                                   : 0u) ^ 0x80808080u);
        }
        // the newest frames of SPB spectra, one batch ahead, 16-byte copies
        // (sub-band input: 4-byte copies of this band's samples, nsub words apart)
        auto stage = [&](int sb, int buf) {
            const int nbb = min(SPB, s_end - sb);
            if (p.nsub > 1) {
                for (int e = t; e < nbb * PTS; e += PTS) {
                    const int u = e / PTS, r = e % PTS;  // r = n2 C + c
                    const long long fr = s0 + sb + u + p.P - 1;
                    const uint32_t *src = reinterpret_cast<const uint32_t *>(p.in) +
                                          (fr * p.N + n1_0 + (long long)p.N1 * (r / C) + r % C) * p.nsub + band;
                    uint32_t *dst = raw + (buf * SPB + u) * PTS + r;
                    if (dbg_ok(fr < p.nframes, kDbgInput))
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;"
                                     :: "r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
                return;
            }
            constexpr int per_row = C / 4, per_frame = PTS / 4;
            for (int e = t; e < nbb * per_frame; e += PTS) {
                const int u = e / per_frame, r = e % per_frame;
                const int n2 = r / per_row, ch = r % per_row;
                const long long fr = s0 + sb + u + p.P - 1;
                const uint32_t *src = reinterpret_cast<const uint32_t *>(p.in) + fr * p.N + n1_0 +
                                      (long long)p.N1 * n2 + ch * 4;
                uint32_t *dst = raw + (buf * SPB + u) * PTS + n2 * C + ch * 4;
                if (dbg_ok(fr < p.nframes, kDbgInput))
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                                 :: "r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        stage(s_beg, 0);
        for (int s_base = s_beg, buf = 0; s_base < s_end; s_base += SPB, buf ^= 1) {
            const int nb = min(SPB, s_end - s_base);
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncthreads();  // frames visible; the other buffer and data are free
            if (s_base + SPB < s_end) stage(s_base + SPB, buf ^ 1);
            float2 cf2[PT];
#pragma unroll
            for (int k = 0; k < PT; k++) cf2[k] = dup2(cfs[k * PTS + t]);
            auto fir_one = [&](auto uc) {
                constexpr int u = decltype(uc)::value;
                constexpr int snew = (u + PT - 1) % PT;
                win[snew] = unpack_p2(raw[(buf * SPB + u) * PTS + t] ^ 0x80808080u);
                const P2 &w0 = win[u % PT];
                P2 y{__fmul2_rn(cf2[0], w0.re), __fmul2_rn(cf2[0], w0.im)};
#pragma unroll
                for (int k = 1; k < PT; k++) {
                    const P2 &wk = win[(u + k) % PT];
                    y.re = __ffma2_rn(cf2[k], wk.re, y.re);
                    y.im = __ffma2_rn(cf2[k], wk.im, y.im);
                }
                data[u * SS + G::pad(t)] = y;
            };
            if (nb == SPB) for_slots(fir_one, std::make_integer_sequence<int, SPB>{});
            else for_slots_below(fir_one, nb, std::make_integer_sequence<int, SPB>{});
            __syncthreads();  // the batch's pre-filter outputs are in data
            if constexpr (G::kOnePass) {
#pragma unroll
                for (int k = 0; k < G::CPT; k++) {
                    const int col = t + k * PTS;  // = sb * C + c
                    const int sb = col / C, c = col % C;
                    if (sb < nb) {
                        P2 v[N2];
#pragma unroll
                        for (int q = 0; q < N2; q++) v[q] = data[sb * SS + q * C + c];
                        Dft<N2>::run(v);
                        P2 *z = reinterpret_cast<P2 *>(Zc) + (size_t)(s_base + sb) * zs + n1_0 + c;
                        if (!dbg_ok(s_base + sb < sc && n1_0 + c < p.N1, kDbgScratch)) continue;
                        z[0] = v[0];
#pragma unroll
                        for (int q = 1; q < N2; q++) z[(size_t)q * p.N1] = cmul(v[q], tws[G::twi(q, c)]);
                    }
                }
            } else {
                constexpr int M1 = N2 / R1, R2 = G::R2;
                // first pass: butterfly j of column (sb, c) over positions j + M1 q
#pragma unroll
                for (int k = 0; k < G::B1; k++) {
                    const int e = t + k * PTS;
                    const int c = e % C, j = (e / C) % M1, sb = e / (C * M1);
                    if (sb < nb) {
                        P2 *d = data + sb * SS + j * C + c;  // + pad((j C + c) + q M1 C) - (j C + c)
                        P2 v[R1];
#pragma unroll
                        for (int q = 0; q < R1; q++) v[q] = d[G::pad(q * M1 * C)];
                        Dft<R1>::run(v);
                        const float2 *w = twc + j * (R1 - 1);
                        d[0] = v[0];
#pragma unroll
                        for (int q = 1; q < R1; q++) d[G::pad(q * M1 * C)] = cmul(v[q], w[q - 1]);
                    }
                }
                __syncthreads();
                // second pass: block b of column (sb, c), positions b R2 + q, to the scratch
#pragma unroll
                for (int k = 0; k < G::B2; k++) {
                    const int e = t + k * PTS;
                    const int c = e % C, b = (e / C) % R1, sb = e / (C * R1);
                    if (sb < nb) {
                        const P2 *d = data + sb * SS + G::pad(b * R2 * C) + c;
                        P2 v[R2];
#pragma unroll
                        for (int q = 0; q < R2; q++) v[q] = d[q * C];
                        Dft<R2>::run(v);
                        P2 *z = reinterpret_cast<P2 *>(Zc) + (size_t)(s_base + sb) * zs +
                                (size_t)(b * R2) * p.N1 + n1_0 + c;
                        if (!dbg_ok(s_base + sb < sc && n1_0 + c < p.N1, kDbgScratch)) continue;
#pragma unroll
                        for (int q = 0; q < R2; q++) z[(size_t)q * p.N1] = cmul(v[q], tws[G::twi(b * R2 + q, c)]);
                    }
                }
            }
        }
        __syncthreads();  // the column passes are done with the twiddle tile
    }
}

template <int N2, int R1 = N2>
__global__ void __launch_bounds__(512, 1) fir_colreg_kernel(const __grid_constant__ ColParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const TileSplit sp = tile_split(p.tiles, p.sc, p.G);
    bool first = true;
    for (long long f = sp.lo; f < sp.hi;) {
        const long long base = f / p.sc * p.sc;  // first item of this super-tile
        const int x = (int)(f / p.sc) * sp.G + sp.r;
        const int s_beg = (int)(f - base);
        const int s_end = (int)(min(sp.hi, base + p.sc) - base);
        f = base + s_end;
        if (p.band < 0) {  // every band in this launch: adjacent tiles are the bands of one column tile
            const int band = x % p.nsub;
            colreg_tile<N2, R1>(p, reinterpret_cast<P2 *>(p.Z) + (size_t)band * p.N, p.s0, p.sc, x / p.nsub, s_beg,
                                s_end, smem_raw, first, band);
        } else {
            colreg_tile<N2, R1>(p, p.Z, p.s0, p.sc, x, s_beg, s_end, smem_raw, first, p.band);
        }
        first = false;
    }
}

// Kernel A, register-column form for dual-pol direct FFT (no pre-filter):
// tiles of C = 2048 / N2 columns, N2 = 2 .. 256. SPB spectra per batch; their
// int8 frames are staged into shared memory one batch ahead. Columns of at
// most 16 points are whole DFTs in registers straight from the staged bytes
// (one pass, natural output order); longer columns take two DIF passes,
// radix 16 then N2 / 16 (the plan's column pass list {16, N2/16}): the first
// reads the staged bytes and writes fp32 to shared memory, the second writes
// the chunk scratch. Every output is multiplied by W_N^(n1 k2) on its way out.
template <int N2>
struct ColDir {
    static constexpr int PTS = 2048, C = PTS / N2, SPB = 4;
    static constexpr bool kOnePass = N2 <= 16;
    static constexpr int R1 = kOnePass ? N2 : 16, R2 = N2 / R1, M1 = N2 / R1;
    static constexpr int CPT = SPB * C / 512;                // columns per thread (one pass)
    static constexpr int B1 = SPB * C * M1 / 512;            // first-pass butterflies per thread
    static constexpr int B2 = SPB * C * R1 / 512;            // second-pass butterflies per thread
    static constexpr int TWC = kOnePass ? 0 : M1 * (R1 - 1);  // first-pass twiddles
    // raw frames [2][SPB][PTS] u32, data [SPB][PTS] P2 (two-pass form),
    // twiddle tile [N2][C] float2, first-pass twiddles [TWC] float2, window
    // values of the tile [N2][C] float
    static constexpr size_t smem = 2 * (size_t)SPB * PTS * 4 + (kOnePass ? 0 : (size_t)SPB * PTS * 16) +
                                   (size_t)PTS * 8 + (size_t)TWC * 8 + (size_t)PTS * 4;
    static_assert(N2 >= 2 && N2 <= 256 && C >= 8, "column shapes of this kernel");
};

// Tile x of the direct-mode register-column kernel A over spectra s_beg ..
// s_end - 1 of a chunk: spectrum s of the chunk is absolute spectrum s0 + s
// and goes to Zc[s] (the chunk holds sc spectra). All 512 threads of the CTA
// take part; the function ends with a barrier. load_twc: load the first-pass
// twiddles (they stay in shared memory for later tiles of the same launch).
template <int N2>
__device__ __forceinline__ void coldir_tile(const ColParams &p, void *Zc, long long s0, int sc, int x, int s_beg,
                                            int s_end, unsigned char *smem_raw, bool load_twc, int band = 0) {
    using G = ColDir<N2>;
    constexpr int PTS = G::PTS, C = G::C, SPB = G::SPB, R1 = G::R1, R2 = G::R2, M1 = G::M1;
    uint32_t *raw = reinterpret_cast<uint32_t *>(smem_raw);                        // [2][SPB][PTS]
    P2 *data = reinterpret_cast<P2 *>(raw + 2 * SPB * PTS);                        // [SPB][PTS]
    float2 *tws = reinterpret_cast<float2 *>(data + (G::kOnePass ? 0 : SPB * PTS));  // [N2][C]
    float2 *twc = tws + PTS;                                                       // [M1][R1-1]
    float *wins = reinterpret_cast<float *>(twc + G::TWC);                         // [N2][C]
    const int t = threadIdx.x;
    const size_t zs = p.zstride > 0 ? (size_t)p.zstride : (size_t)p.N;  // scratch spectrum stride
    if (load_twc)
        for (int e = t; e < G::TWC; e += 512) twc[e] = __ldg(p.twA + p.pass[0].off + e);
    // sample (pos e of the tile) of spectrum row rb, times the window value when there is one
    auto sample = [&](const uint32_t *rb, int e) {
        P2 v = unpack_p2(rb[e] ^ 0x80808080u);
        if (p.win) {
            const float2 h = dup2(wins[e]);
            v = P2{__fmul2_rn(v.re, h), __fmul2_rn(v.im, h)};
        }
        return v;
    };
    {
        const int n1_0 = x * C;
        for (int e = t; e < PTS; e += 512) {  // W_N^(n1 k2(pos)); window values h[n1 + N1 n2]
            tws[e] = __ldg(p.twZ + (size_t)(e / C) * p.N1 + n1_0 + (e % C));
            if (p.win) wins[e] = __ldg(p.coef + (size_t)(e / C) * p.N1 + n1_0 + (e % C));
        }
        // frames of SPB spectra into raw[buf], 16-byte copies (sub-band input:
        // 4-byte copies of this band's samples, nsub words apart)
        auto stage = [&](int sb, int buf) {
            const int nbb = min(SPB, s_end - sb);
            if (p.nsub > 1) {
                for (int e = t; e < nbb * PTS; e += 512) {
                    const int u = e / PTS, r = e % PTS;  // r = n2 C + c
                    const long long fr = s0 + sb + u;
                    const uint32_t *src = reinterpret_cast<const uint32_t *>(p.in) +
                                          (fr * p.N + n1_0 + (long long)p.N1 * (r / C) + r % C) * p.nsub + band;
                    uint32_t *dst = raw + (buf * SPB + u) * PTS + r;
                    if (dbg_ok(fr < p.nframes, kDbgInput))
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;"
                                     :: "r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
                return;
            }
            constexpr int per_row = C / 4, per_frame = PTS / 4;
            for (int e = t; e < nbb * per_frame; e += 512) {
                const int u = e / per_frame, r = e % per_frame;
                const int n2 = r / per_row, ch = r % per_row;
                const long long fr = s0 + sb + u;
                const uint32_t *src = reinterpret_cast<const uint32_t *>(p.in) + fr * p.N + n1_0 +
                                      (long long)p.N1 * n2 + ch * 4;
                uint32_t *dst = raw + (buf * SPB + u) * PTS + n2 * C + ch * 4;
                if (dbg_ok(fr < p.nframes, kDbgInput))
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                                 :: "r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        stage(s_beg, 0);
        for (int s_base = s_beg, buf = 0; s_base < s_end; s_base += SPB, buf ^= 1) {
            const int nb = min(SPB, s_end - s_base);
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncthreads();  // frames and the twiddle tile visible; the other buffer and data are free
            if (s_base + SPB < s_end) stage(s_base + SPB, buf ^ 1);
            const uint32_t *rb = raw + buf * SPB * PTS;
            if constexpr (G::kOnePass) {
#pragma unroll
                for (int k = 0; k < G::CPT; k++) {
                    const int col = t + k * 512;  // = sb * C + c
                    const int sb = col / C, c = col % C;
                    if (sb < nb) {
                        P2 v[N2];
#pragma unroll
                        for (int q = 0; q < N2; q++) v[q] = sample(rb + sb * PTS, q * C + c);
                        Dft<N2>::run(v);
                        P2 *z = reinterpret_cast<P2 *>(Zc) + (size_t)(s_base + sb) * zs + n1_0 + c;
                        if (!dbg_ok(s_base + sb < sc && n1_0 + c < p.N1, kDbgScratch)) continue;
                        z[0] = v[0];
#pragma unroll
                        for (int q = 1; q < N2; q++) z[(size_t)q * p.N1] = cmul(v[q], tws[q * C + c]);
                    }
                }
            } else {
                // first pass: butterfly j of column (sb, c) over positions j + M1 q
#pragma unroll
                for (int k = 0; k < G::B1; k++) {
                    const int e = t + k * 512;
                    const int c = e % C, j = (e / C) % M1, sb = e / (C * M1);
                    if (sb < nb) {
                        const int o = sb * PTS + j * C + c;
                        P2 v[R1];
#pragma unroll
                        for (int q = 0; q < R1; q++) v[q] = sample(rb + sb * PTS, (j + q * M1) * C + c);
                        Dft<R1>::run(v);
                        const float2 *w = twc + j * (R1 - 1);
                        data[o] = v[0];
#pragma unroll
                        for (int q = 1; q < R1; q++) data[o + q * M1 * C] = cmul(v[q], w[q - 1]);
                    }
                }
                __syncthreads();
                // second pass: block b of column (sb, c), positions b R2 + q, to the scratch
#pragma unroll
                for (int k = 0; k < G::B2; k++) {
                    const int e = t + k * 512;
                    const int c = e % C, b = (e / C) % R1, sb = e / (C * R1);
                    if (sb < nb) {
                        const P2 *d = data + sb * PTS + b * R2 * C + c;
                        P2 v[R2];
#pragma unroll
                        for (int q = 0; q < R2; q++) v[q] = d[q * C];
                        Dft<R2>::run(v);
                        P2 *z = reinterpret_cast<P2 *>(Zc) + (size_t)(s_base + sb) * zs +
                                (size_t)(b * R2) * p.N1 + n1_0 + c;
                        if (!dbg_ok(s_base + sb < sc && n1_0 + c < p.N1, kDbgScratch)) continue;
#pragma unroll
                        for (int q = 0; q < R2; q++) z[(size_t)q * p.N1] = cmul(v[q], tws[(b * R2 + q) * C + c]);
                    }
                }
            }
        }
        __syncthreads();  // the column passes are done with the twiddle tile and data
    }
}

template <int N2>
__global__ void __launch_bounds__(512) fir_coldir_kernel(const __grid_constant__ ColParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const TileSplit sp = tile_split(p.tiles, p.sc, p.G);
    bool first = true;
    for (long long f = sp.lo; f < sp.hi;) {
        const long long base = f / p.sc * p.sc;  // first item of this super-tile
        const int x = (int)(f / p.sc) * sp.G + sp.r;
        const int s_beg = (int)(f - base);
        const int s_end = (int)(min(sp.hi, base + p.sc) - base);
        f = base + s_end;
        if (p.band < 0) {  // every band in this launch: adjacent tiles are the bands of one column tile
            const int band = x % p.nsub;
            coldir_tile<N2>(p, reinterpret_cast<P2 *>(p.Z) + (size_t)band * p.N, p.s0, p.sc, x / p.nsub, s_beg, s_end,
                            smem_raw, first, band);
        } else {
            coldir_tile<N2>(p, p.Z, p.s0, p.sc, x, s_beg, s_end, smem_raw, first, p.band);
        }
        first = false;
    }
}

// Kernel A for transforms too long for a register FIR window next to the
// column tile (PFB with nchan above 2^18): every spectrum's P taps are read
// straight from the input (the P frames a spectrum spans stay in L2 while
// the block walks its consecutive spectra), the coefficients from L1/L2.
template <int NPOL, int PPT>
__global__ void __launch_bounds__(512) fir_colfft_gather_kernel(const __grid_constant__ ColParams p) {
    using T = typename Elem<NPOL>::T;
    constexpr int NC = 2 * NPOL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *data = reinterpret_cast<T *>(smem_raw);  // [N2][C]
    float2 *tws = reinterpret_cast<float2 *>(data + p.N2 * p.C);  // [N2][C]
    const TileSplit sp = tile_split(p.tiles, p.sc, p.G);
    for (long long f = sp.lo; f < sp.hi;) {
        const long long base = f / p.sc * p.sc;  // first item of this super-tile
        const int x = (int)(f / p.sc) * sp.G + sp.r;
        const int s_beg = (int)(f - base);
        const int s_end = (int)(min(sp.hi, base + p.sc) - base);
        f = base + s_end;
        stage_tile_twiddles(p, tws, x);  // ordered before use by the barrier below
        long long n_pt[PPT];
#pragma unroll
        for (int i = 0; i < PPT; i++) {
            const int idx = threadIdx.x + i * blockDim.x;  // = n2 * C + c
            n_pt[i] = x * p.C + (idx & (p.C - 1)) + (long long)p.N1 * (idx >> p.lC);
        }
        for (int s = s_beg; s < s_end; s++) {
            const long long f0 = p.s0 + s;  // oldest frame of spectrum s
            float y[PPT][NC];
#pragma unroll
            for (int i = 0; i < PPT; i++)
#pragma unroll
                for (int k = 0; k < NC; k++) y[i][k] = 0.f;
#pragma unroll 4
            for (int t = 0; t < p.P; t++) {
#pragma unroll
                for (int i = 0; i < PPT; i++) {
                    const float c = __ldg(p.coef + (size_t)t * p.N + n_pt[i]);
                    const uint32_t wx = load_raw<NPOL>(p.in, (f0 + t) * p.N + n_pt[i]) ^ 0x80808080u;
#pragma unroll
                    for (int k = 0; k < NC; k++) y[i][k] = fmaf(c, unpack_byte(wx, k), y[i][k]);
                }
            }
#pragma unroll
            for (int i = 0; i < PPT; i++) {
                T *d = data + threadIdx.x + i * blockDim.x;
                if constexpr (NPOL == 2) *d = make_p2(y[i][0], y[i][1], y[i][2], y[i][3]);
                else *d = make_float2(y[i][0], y[i][1]);
            }
            __syncthreads();
            // ends on a barrier: data is free for the next spectrum
            col_fft_store<NPOL, col_radix_cap(NPOL, 1, PPT)>(p, data, x, s, 1, tws);
        }
    }
}

// ---------------------------------------------------------------- kernel B --

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

template <int NPOL> __device__ __forceinline__ void acc_add(float4 &a, float4 v) {
    // detection of one channel of both polarisations (§4)
    const float xx = fmaf(v.x, v.x, v.y * v.y);
    const float yy = fmaf(v.z, v.z, v.w * v.w);
    const float re = fmaf(v.x, v.z, v.y * v.w);   // Re(X conj Y)
    const float im = fmaf(v.y, v.z, -v.x * v.w);  // Im(X conj Y)
    a.x += xx;
    a.y += yy;
    a.z += re;
    a.w += im;
}
// the same from the packed form: (XX, YY) is one paired operation
__device__ __forceinline__ float4 detect4(P2 v) {
    const float2 p = __ffma2_rn(v.re, v.re, __fmul2_rn(v.im, v.im));  // (|X|^2, |Y|^2)
    return make_float4(p.x, p.y, fmaf(v.re.x, v.re.y, v.im.x * v.im.y), fmaf(v.im.x, v.re.y, -(v.re.x * v.im.y)));
}
// a += detect4(v), each product accumulated by a fused multiply-add
// (|X|^2 and |Y|^2 as one pair)
template <int NPOL> __device__ __forceinline__ void acc_add(float4 &a, P2 v) {
    float2 xy = __ffma2_rn(v.im, v.im, make_float2(a.x, a.y));
    xy = __ffma2_rn(v.re, v.re, xy);
    a.x = xy.x;
    a.y = xy.y;
    a.z = fmaf(v.re.x, v.re.y, fmaf(v.im.x, v.im.y, a.z));
    a.w = fmaf(v.im.x, v.re.y, fmaf(-v.re.x, v.im.y, a.w));
}
__device__ __forceinline__ void acc_add1(float &a, float2 v) { a += fmaf(v.x, v.x, v.y * v.y); }

// Compensated (Kahan) summation a += v with running compensation c.
__device__ __forceinline__ void kahan_add(float &a, float &c, float v) {
    const float y = v - c;
    const float t = a + y;
    c = (t - a) - y;
    a = t;
}
__device__ __forceinline__ void kahan_add(float4 &a, float4 &c, float4 v) {
    kahan_add(a.x, c.x, v.x);
    kahan_add(a.y, c.y, v.y);
    kahan_add(a.z, c.z, v.z);
    kahan_add(a.w, c.w, v.w);
}
// Fold the compensation into the value (Fast2Sum, exact since |c| <= |a|):
// afterwards a is the correctly rounded a - c and a - c is unchanged.
__device__ __forceinline__ void kahan_settle(float &a, float &c) {
    const float t = a - c;
    c = (t - a) + c;
    a = t;
}
__device__ __forceinline__ void kahan_settle(float4 &a, float4 &c) {
    kahan_settle(a.x, c.x);
    kahan_settle(a.y, c.y);
    kahan_settle(a.z, c.z);
    kahan_settle(a.w, c.w);
}
__device__ __forceinline__ float4 detect4(float4 v) {
    return make_float4(fmaf(v.x, v.x, v.y * v.y), fmaf(v.z, v.z, v.w * v.w), fmaf(v.x, v.z, v.y * v.w),
                       fmaf(v.y, v.z, -v.x * v.w));
}
__device__ __forceinline__ float4 sub4(float4 a, float4 b) {
    return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}

// Pre-filter output y_s[n] = sum_t h[t N + n] x[(s + t) N + n] of one sample
// (h[0] on the oldest frame), straight from the int8 input.
template <int NPOL>
__device__ __forceinline__ typename Elem<NPOL>::T fir_sample(const RowParams &p, long long sabs, int n) {
    constexpr int NC = 2 * NPOL;
    float a[NC];
#pragma unroll
    for (int k = 0; k < NC; k++) a[k] = 0.f;
    for (int t = 0; t < p.P; t++) {
        const float c = __ldg(p.coef + (size_t)t * p.N + n);
        const uint32_t w = load_raw<NPOL>(p.in, (sabs + t) * p.N + n) ^ 0x80808080u;
#pragma unroll
        for (int k = 0; k < NC; k++) a[k] = fmaf(c, unpack_byte(w, k), a[k]);
    }
    if constexpr (NPOL == 2) return make_p2(a[0], a[1], a[2], a[3]);
    else return make_float2(a[0], a[1]);
}

// The same pre-filter output from frames staged in shared memory: ring slot
// (slot0 + t) mod (P + 1) holds frame s + t as int8 (N1 samples), cfs[t N1 + n]
// the coefficients h[t N + n] (one-row transforms, N = N1).
template <int NPOL>
__device__ __forceinline__ typename Elem<NPOL>::T fir_ring(const unsigned char *ring, const float *cfs, int N1,
                                                           int P, int slot0, int n) {
    constexpr int NC = 2 * NPOL;
    float a[NC];
#pragma unroll
    for (int k = 0; k < NC; k++) a[k] = 0.f;
    int slot = slot0;
    for (int t = 0; t < P; t++) {
        const float c = cfs[t * N1 + n];
        uint32_t w;
        if constexpr (NPOL == 2) w = reinterpret_cast<const uint32_t *>(ring)[slot * N1 + n];
        else w = reinterpret_cast<const unsigned short *>(ring)[slot * N1 + n];
        w ^= 0x80808080u;
#pragma unroll
        for (int k = 0; k < NC; k++) a[k] = fmaf(c, unpack_byte(w, k), a[k]);
        slot = slot == P ? 0 : slot + 1;
    }
    if constexpr (NPOL == 2) return make_p2(a[0], a[1], a[2], a[3]);
    else return make_float2(a[0], a[1]);
}

constexpr int kRowRun = 16;  // spectra per accumulator run of the general row kernel

template <int R, int NPOL, bool KAHAN = false, bool FIR = false>
__device__ __forceinline__ void row_butterfly(const RowParams &p, int x, typename Elem<NPOL>::T *data,
                                              typename Elem<NPOL>::Acc *acc,
                                              const typename Elem<NPOL>::T *Zs, const Pass ps,
                                              bool first, bool last, int r, int b, int j,
                                              int rowstride, typename Elem<NPOL>::Acc *comp = nullptr,
                                              const unsigned char *ring = nullptr, const float *cfs = nullptr,
                                              int slot0 = 0) {
    using T = typename Elem<NPOL>::T;
    const int base = b * ps.lb + j;
    T *row = data + r * rowstride;
    T v[R];
    if (FIR && first) {
#pragma unroll
        for (int q = 0; q < R; q++) v[q] = fir_ring<NPOL>(ring, cfs, p.N1, p.P, slot0, base + q * ps.m);
    } else if (first) {
        const T *zr = Zs + (size_t)(x * p.RB + r) * p.N1;
#pragma unroll
        for (int q = 0; q < R; q++) v[q] = ld_no_l1(zr + base + q * ps.m);  // read once
    } else {
#pragma unroll
        for (int q = 0; q < R; q++) v[q] = row[pad16(base + q * ps.m)];
    }
    Dft<R>::run(v);
    if (!last) {
        if (ps.m > 1) {
            const float2 *tw = p.twB + ps.off + j * (R - 1);
#pragma unroll
            for (int q = 1; q < R; q++) v[q] = cmul(v[q], __ldg(tw + q - 1));
        }
#pragma unroll
        for (int q = 0; q < R; q++) row[pad16(base + q * ps.m)] = v[q];
    } else {
        // m == 1: output q of unit (r, b); accumulator slot q * U + (r * N1/R + b)
        constexpr int LR = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
        const int U = p.RB << (p.lN1 - LR);
        const int w = (r << (p.lN1 - LR)) + b;
#pragma unroll
        for (int q = 0; q < R; q++) {
            if constexpr (KAHAN) {
                if constexpr (NPOL == 2) kahan_add(acc[q * U + w], comp[q * U + w], detect4(v[q]));
                else kahan_add(acc[q * U + w], comp[q * U + w], fmaf(v[q].x, v[q].x, v[q].y * v[q].y));
            } else {
                if constexpr (NPOL == 2) acc_add<2>(acc[q * U + w], v[q]);
                else acc_add1(acc[q * U + w], v[q]);
            }
        }
    }
}

// Shared memory of the general row kernel: RB padded rows, the accumulators
// (and their compensation), then, for one-row transforms, the frame ring and
// coefficients at a 16-byte boundary.
template <int NPOL, bool KAHAN>
__host__ __device__ constexpr size_t row_ring_offset(int RB, int N1) {
    return ((size_t)RB * (N1 + (N1 >> 4)) * sizeof(typename Elem<NPOL>::T) +
            (size_t)RB * N1 * sizeof(typename Elem<NPOL>::Acc) * (KAHAN ? 2 : 1) + 15) & ~(size_t)15;
}
__host__ __device__ constexpr size_t row_ring_bytes(int npol, int P, int N1) {
    return (size_t)(P + 1) * N1 * 2 * npol + (size_t)P * N1 * 4;
}

template <int NPOL, bool KAHAN = false, bool FIR = false>
__global__ void __launch_bounds__(256, 2) rowfft_detect_kernel(const __grid_constant__ RowParams p) {
    using T = typename Elem<NPOL>::T;
    using A = typename Elem<NPOL>::Acc;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int rowstride = p.N1 + (p.N1 >> 4);
    T *data = reinterpret_cast<T *>(smem_raw);
    A *acc = reinterpret_cast<A *>(data + p.RB * rowstride);
    A *comp = acc + p.RB * p.N1;  // compensation (compensated plans only)
    const int nacc = p.RB * p.N1;
    const int RL = p.pass[p.npass - 1].r;
    const int lq = p.lN1 - p.pass[p.npass - 1].lr;  // log2 (N1 / RL)
    const int lU = p.lRB + lq;
    // one-row transforms (FIR): a ring of P + 1 int8 frames and the P taps'
    // coefficients in shared memory, filled with 16-byte asynchronous copies;
    // the frame of the next spectrum is copied while this one is transformed
    constexpr int W = 2 * NPOL;  // bytes per sample
    unsigned char *ring = smem_raw + row_ring_offset<NPOL, KAHAN>(p.RB, p.N1);
    float *cfs = reinterpret_cast<float *>(ring + (FIR ? (size_t)(p.P + 1) * p.N1 * W : 0));
    auto copy16 = [&](void *dst, const void *src, int bytes) {
        for (int e = threadIdx.x; e < bytes / 16; e += blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                         :: "r"((uint32_t)__cvta_generic_to_shared(static_cast<unsigned char *>(dst) + 16 * e)),
                            "l"(static_cast<const unsigned char *>(src) + 16 * e) : "memory");
    };
    auto stage_frame = [&](long long fr) {  // frame fr into slot fr mod (P + 1)
        copy16(ring + (size_t)(fr % (p.P + 1)) * p.N1 * W, p.in + fr * p.N * W, p.N1 * W);
    };
    if constexpr (FIR) copy16(cfs, p.coef, p.P * p.N1 * 4);

    const Span sp = block_span(p.tiles, p.sc);
    for (long long f = sp.lo; f < sp.hi;) {
        const int x = (int)(f / p.sc);  // row tile
        const long long base = (long long)x * p.sc;
        const int s_beg = (int)(f - base);
        const int s_end = (int)(min(sp.hi, base + p.sc) - base);
        f = base + s_end;

        for (int e = threadIdx.x; e < nacc; e += blockDim.x) {
            if constexpr (NPOL == 2) acc[e] = make_float4(0.f, 0.f, 0.f, 0.f);
            else acc[e] = 0.f;
            if constexpr (KAHAN) comp[e] = acc[e];
        }
        // add the accumulators into this block's slot: accumulator e = q * U +
        // (r * N1/R + b) holds row r, position b*R + q; `store`: the slot's
        // first write this call. Each thread flushes the entries it zeroes.
        auto flush = [&](bool store) {
            const size_t so = (size_t)span_slot(p.tiles, p.sc, x) * p.N;
            A *part = reinterpret_cast<A *>(p.partial) + so;
            const bool slot_ok = dbg_ok(span_slot(p.tiles, p.sc, x) < p.slots && x < p.tiles, kDbgSlot);
            for (int e = threadIdx.x; e < nacc && slot_ok; e += blockDim.x) {
                const int q = e >> lU, w = e & ((1 << lU) - 1);
                const int r = w >> lq, b = w & ((1 << lq) - 1);
                const size_t o = (size_t)(x * p.RB + r) * p.N1 + b * RL + q;
                if constexpr (KAHAN) {
                    A *pc = reinterpret_cast<A *>(p.partial_comp) + so;
                    A a = part[o], c = pc[o];
                    if constexpr (NPOL == 2) kahan_add(a, c, sub4(acc[e], comp[e]));
                    else kahan_add(a, c, acc[e] - comp[e]);
                    part[o] = a;
                    pc[o] = c;
                } else if (store) {
                    part[o] = acc[e];
                } else {
                    atomicAdd(part + o, acc[e]);  // in L2, one writer per entry (see row2048_kernel)
                }
            }
        };
        bool first = p.store != 0;
        if constexpr (FIR) {  // the segment's first spectrum's P frames
            for (int t = 0; t < p.P; t++) stage_frame(p.s0 + s_beg + t);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        __syncthreads();

        for (int s = s_beg; s < s_end; s++) {
            const T *Zs = FIR ? nullptr : reinterpret_cast<const T *>(p.Z) + (size_t)s * p.N;
            if constexpr (FIR) {
                // the next spectrum's newest frame takes the slot of frame s - 1,
                // which the previous spectrum's passes are done with
                if (s + 1 < s_end) {
                    stage_frame(p.s0 + s + p.P);
                    asm volatile("cp.async.commit_group;" ::: "memory");
                    asm volatile("cp.async.wait_group 1;" ::: "memory");
                } else {
                    asm volatile("cp.async.wait_group 0;" ::: "memory");
                }
                __syncthreads();  // spectrum s's frames are visible to every thread
            }
            const int slot0 = FIR ? (int)((p.s0 + s) % (p.P + 1)) : 0;
            for (int ip = 0; ip < p.npass; ip++) {
                const Pass ps = p.pass[ip];
                const bool first = ip == 0, last = ip == p.npass - 1;
                const int lper = p.lN1 - ps.lr;  // log2 butterflies per row
                const int nb = p.RB << lper;
                for (int u = threadIdx.x; u < nb; u += blockDim.x) {
                    const int r = u >> lper, w = u & ((1 << lper) - 1);
                    const int b = w >> ps.lm, j = w & (ps.m - 1);
                    switch (ps.r) {
                        case 2: row_butterfly<2, NPOL, KAHAN, FIR>(p, x, data, acc, Zs, ps, first, last, r, b, j, rowstride, comp, ring, cfs, slot0); break;
                        case 4: row_butterfly<4, NPOL, KAHAN, FIR>(p, x, data, acc, Zs, ps, first, last, r, b, j, rowstride, comp, ring, cfs, slot0); break;
                        case 8: row_butterfly<8, NPOL, KAHAN, FIR>(p, x, data, acc, Zs, ps, first, last, r, b, j, rowstride, comp, ring, cfs, slot0); break;
                        default: row_butterfly<16, NPOL, KAHAN, FIR>(p, x, data, acc, Zs, ps, first, last, r, b, j, rowstride, comp, ring, cfs, slot0); break;
                    }
                }
                __syncthreads();
            }
            // uncompensated sums: after a run of kRowRun spectra with more to
            // come, into the slot (two-level summation, as in the 2048-point
            // kernel); the barrier orders the zeroing before the next
            // spectrum's last pass adds again (a one-pass row adds in its
            // first pass)
            if constexpr (!KAHAN) {
                if ((s - s_beg) % kRowRun == kRowRun - 1 && s + 1 < s_end) {
                    flush(first);
                    first = false;
                    for (int e = threadIdx.x; e < nacc; e += blockDim.x) {
                        if constexpr (NPOL == 2) acc[e] = make_float4(0.f, 0.f, 0.f, 0.f);
                        else acc[e] = 0.f;
                    }
                    __syncthreads();
                }
            }
        }

        flush(first);
        __syncthreads();  // acc is zeroed again by the next segment
    }
}

// ------------------------------------------------------ kernel B, 2048 --
// Rows of 2048 points (RB = 1; passes radix 16, 16, 8), two spectra at a
// time. In the radix-16 passes (128 butterflies each) the block's halves
// transform one spectrum each, synchronising on their own named barrier;
// the radix-8 pass (256 butterflies) then runs over both spectra with every
// thread. Thread t always computes outputs 8t .. 8t+7 of the last pass, so
// its eight channels' accumulators live in registers. Rows are stored with
// one pad element every 8 (pad8), which keeps all three passes' accesses
// free of bank conflicts.
//
// Uncompensated plans sum in two levels: the registers take a run of
// kRow2048Run spectra, then the run's sums are added into the CTA's
// partial-sum slot (in L2) and the registers restart from zero. A segment of
// S spectra then makes runs of kRow2048Run additions and S / kRow2048Run
// additions of run sums instead of one chain of S additions, which cuts the
// FP32 summation error of long segments (hundreds of spectra per CTA on the
// long workloads) by about the square root of the run length, for one
// reduction into L2 of the thread's eight channels per run.
__device__ __forceinline__ int pad8(int i) { return i + (i >> 3); }
constexpr int kRow2048Stride = 2048 + 2048 / 8;
constexpr int kRow2048Run = 16;  // spectra per register run (a multiple of 2)

// Barriers of a 2048-point row worker of 256 threads: the whole CTA (the
// ordinary kernel), or one of the two 256-thread groups of a 512-thread CTA
// (named barriers 1 + g for the group, 3 + 2 g + half for its halves).
struct RowGrpCta {
    __device__ __forceinline__ int tid() const { return threadIdx.x; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ void sync_half(int half) const {
        if (half) asm volatile("bar.sync 2, 128;" ::: "memory");
        else asm volatile("bar.sync 1, 128;" ::: "memory");
    }
};
struct RowGrp2 {
    int g;  // threads 256 g .. 256 g + 255
    __device__ __forceinline__ int tid() const { return threadIdx.x & 255; }
    __device__ __forceinline__ void sync() const { asm volatile("bar.sync %0, 256;" :: "r"(1 + g) : "memory"); }
    __device__ __forceinline__ void sync_half(int half) const {
        asm volatile("bar.sync %0, 128;" :: "r"(3 + 2 * g + half) : "memory");
    }
};

// ZSPLIT: the scratch elements hold (X.re, X.im, Y.re, Y.im) (the tensor-core
// column kernel's order) instead of the packed (X.re, Y.re, X.im, Y.im).
// RING: the chunk's scratch is Zc (sc spectra), read through L2 only (ld.cg:
// the persistent form rewrites it while CTAs run); otherwise p.Z and p.sc.
template <int NPOL, bool KAHAN, bool FIR, bool ZSPLIT, bool RING, typename GRP>
__device__ __forceinline__ void row2048_first(const RowParams &p, const void *Zc_ring, int sc_ring,
                                              typename Elem<NPOL>::T *row, int x, int s, int ht, int half,
                                              GRP grp) {
    using T = typename Elem<NPOL>::T;
    const void *Zc = RING ? Zc_ring : p.Z;
    const int sc = RING ? sc_ring : p.sc;
    // pass 1: block length 2048, butterfly j = ht over positions j + 128 q
    {
        const Pass ps = p.pass[0];
        T v[16];
        if constexpr (FIR) {
#pragma unroll
            for (int q = 0; q < 16; q++) v[q] = fir_sample<NPOL>(p, p.s0 + s, ht + 128 * q);
        } else if constexpr (ZSPLIT) {
            // the scratch is read once: loads that do not allocate in L1, so
            // that the rows do not push the twiddles out of it
            const float4 *zr = reinterpret_cast<const float4 *>(Zc) + (size_t)s * p.N + (size_t)x * 2048;
#pragma unroll
            for (int q = 0; q < 16; q++) {
                const float4 e = ld_no_l1(zr + ht + 128 * q);
                v[q] = make_p2(e.x, e.y, e.z, e.w);
            }
        } else if (dbg_ok(s < sc && (x + 1) * 2048 <= p.N, kDbgScratch | kDbgTile)) {
            const T *zr = reinterpret_cast<const T *>(Zc) + (size_t)s * p.N + (size_t)x * 2048;
            if constexpr (RING && NPOL == 2) {
                const float4 *z4 = reinterpret_cast<const float4 *>(zr);
#pragma unroll
                for (int q = 0; q < 16; q++) {
                    const float4 e = __ldcg(z4 + ht + 128 * q);
                    v[q] = P2{make_float2(e.x, e.y), make_float2(e.z, e.w)};
                }
            } else if constexpr (NPOL == 2) {
                // read once: loads that do not allocate in L1, so that the
                // rows do not push the twiddles out of it
                const float4 *z4 = reinterpret_cast<const float4 *>(zr);
#pragma unroll
                for (int q = 0; q < 16; q++) {
                    const float4 e = ld_no_l1(z4 + ht + 128 * q);
                    v[q] = P2{make_float2(e.x, e.y), make_float2(e.z, e.w)};
                }
            } else {
#pragma unroll
                for (int q = 0; q < 16; q++) v[q] = zr[ht + 128 * q];
            }
        } else {
#pragma unroll
            for (int q = 0; q < 16; q++) v[q] = T{};
        }
        Dft<16>::run(v);
        const float2 *tw = p.twB + ps.off + ht * 15;
#pragma unroll
        for (int q = 1; q < 16; q++) v[q] = cmul(v[q], __ldg(tw + q - 1));
#pragma unroll
        for (int q = 0; q < 16; q++) row[pad8(ht + 128 * q)] = v[q];
    }
    grp.sync_half(half);
    // pass 2: block length 128, unit b = ht / 8, butterfly j = ht % 8
    {
        const Pass ps = p.pass[1];
        const int b = ht >> 3, j = ht & 7;
        const int base = b * 128 + j;
        T v[16];
#pragma unroll
        for (int q = 0; q < 16; q++) v[q] = row[pad8(base + 8 * q)];
        Dft<16>::run(v);
        const float2 *tw = p.twB + ps.off + j * 15;
#pragma unroll
        for (int q = 1; q < 16; q++) v[q] = cmul(v[q], __ldg(tw + q - 1));
#pragma unroll
        for (int q = 0; q < 16; q++) row[pad8(base + 8 * q)] = v[q];
    }
}

template <int NPOL, bool KAHAN>
__device__ __forceinline__ void row2048_last(const typename Elem<NPOL>::T *row, int t,
                                             typename Elem<NPOL>::Acc (&acc)[8],
                                             typename Elem<NPOL>::Acc (&comp)[8]) {
    using T = typename Elem<NPOL>::T;
    T v[8];
#pragma unroll
    for (int q = 0; q < 8; q++) v[q] = row[pad8(8 * t + q)];
    Dft<8>::run(v);
#pragma unroll
    for (int q = 0; q < 8; q++) {
        if constexpr (KAHAN) {
            if constexpr (NPOL == 2) kahan_add(acc[q], comp[q], detect4(v[q]));
            else kahan_add(acc[q], comp[q], fmaf(v[q].x, v[q].x, v[q].y * v[q].y));
        } else {
            if constexpr (NPOL == 2) acc_add<2>(acc[q], v[q]);
            else acc_add1(acc[q], v[q]);
        }
    }
}

template <int NPOL, bool KAHAN, bool FIR, bool ZSPLIT = false>
__global__ void __launch_bounds__(256, KAHAN ? 1 : 2) row2048_kernel(const __grid_constant__ RowParams p) {
    using T = typename Elem<NPOL>::T;
    using A = typename Elem<NPOL>::Acc;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *rows = reinterpret_cast<T *>(smem_raw);  // two rows, pad8 layout
    const int tid = threadIdx.x, half = tid >> 7, ht = tid & 127;
    T *own = rows + half * kRow2048Stride;

    const Span sp = block_span(p.tiles, p.sc);
    for (long long f = sp.lo; f < sp.hi;) {
        const int x = (int)(f / p.sc);  // row tile
        const long long base = (long long)x * p.sc;
        const int s_beg = (int)(f - base);
        const int s_end = (int)(min(sp.hi, base + p.sc) - base);
        f = base + s_end;

        A acc[8], comp[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            if constexpr (NPOL == 2) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            else acc[q] = 0.f;
            comp[q] = acc[q];
        }
        // add the registers into this block's slot (thread t holds positions
        // 8t .. 8t+7 of row tile x); `store`: the slot's first write this call
        auto flush = [&](bool store) {
            if (!dbg_ok(span_slot(p.tiles, p.sc, x) < p.slots && (x + 1) * 2048 <= p.N, kDbgSlot)) return;
            const size_t so = (size_t)span_slot(p.tiles, p.sc, x) * p.N + (size_t)x * 2048 + 8 * tid;
            A *part = reinterpret_cast<A *>(p.partial) + so;
#pragma unroll
            for (int q = 0; q < 8; q++) {
                if constexpr (KAHAN) {
                    A *pc = reinterpret_cast<A *>(p.partial_comp) + so;
                    A a = part[q], c = pc[q];
                    if constexpr (NPOL == 2) kahan_add(a, c, sub4(acc[q], comp[q]));
                    else kahan_add(a, c, acc[q] - comp[q]);
                    part[q] = a;
                    pc[q] = c;
                } else if (store) {
                    part[q] = acc[q];
                } else {
                    // a reduction performed in L2: no wait for the slot's old
                    // value. Only this thread adds to these entries, in program
                    // order, so the sums are the same as a load-add-store's.
                    atomicAdd(part + q, acc[q]);
                }
            }
        };
        bool first = p.store != 0;
        for (int s = s_beg; s < s_end; s += 2) {
            const bool two = s + 1 < s_end;
            if (half == 0 || two) row2048_first<NPOL, KAHAN, FIR, ZSPLIT, false>(p, nullptr, 0, own, x, s + half, ht, half, RowGrpCta{});
            __syncthreads();
            row2048_last<NPOL, KAHAN>(rows, tid, acc, comp);
            if (two) row2048_last<NPOL, KAHAN>(rows + kRow2048Stride, tid, acc, comp);
            if constexpr (!KAHAN) {
                // end of a register run with more spectra to come: into the slot
                if (((s - s_beg) & (kRow2048Run - 1)) == kRow2048Run - 2 && s + 2 < s_end) {
                    flush(first);
                    first = false;
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        if constexpr (NPOL == 2) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                        else acc[q] = 0.f;
                    }
                }
            }
            __syncthreads();  // both rows are free for the next pair
        }
        flush(first);
    }
}

// Kernel B for 4096-point rows (dual-pol, no pre-filter; 2^19 PFB plans):
// four radix-8 DIF passes over one spectrum's row at a time, 512 threads with
// one butterfly each per pass (pass with block length L: block b, butterfly j
// over positions b L + j + (L / 8) q, outputs times W_L^(j q)). Thread t
// computes outputs 8t .. 8t+7 of the last pass, so its eight channels'
// accumulators stay in registers, with the two-level sums of the 2048-point
// kernel. The row uses the pad8 layout: in every pass the 8 threads of a
// 16-byte phase touch 8 different bank groups.
constexpr int kRow4096Stride = 4096 + 4096 / 8;

template <bool ZSPLIT = false>
__global__ void __launch_bounds__(512, 1) row4096_kernel(const __grid_constant__ RowParams p) {
    using A = float4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    P2 *row = reinterpret_cast<P2 *>(smem_raw);  // one row, pad8 layout
    const int t = threadIdx.x;
    const Span sp = block_span(p.tiles, p.sc);
    for (long long f = sp.lo; f < sp.hi;) {
        const int x = (int)(f / p.sc);  // row tile
        const long long base = (long long)x * p.sc;
        const int s_beg = (int)(f - base);
        const int s_end = (int)(min(sp.hi, base + p.sc) - base);
        f = base + s_end;

        A acc[8];
#pragma unroll
        for (int q = 0; q < 8; q++) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        // add the registers into this block's slot (thread t holds positions
        // 8t .. 8t+7 of row tile x); `store`: the slot's first write this call
        auto flush = [&](bool store) {
            if (!dbg_ok(span_slot(p.tiles, p.sc, x) < p.slots && (x + 1) * 4096 <= p.N, kDbgSlot)) return;
            A *part = reinterpret_cast<A *>(p.partial) + (size_t)span_slot(p.tiles, p.sc, x) * p.N +
                      (size_t)x * 4096 + 8 * t;
#pragma unroll
            for (int q = 0; q < 8; q++) {
                if (store) part[q] = acc[q];
                else atomicAdd(part + q, acc[q]);  // in L2; one writer per entry, in program order
            }
        };
        bool first = p.store != 0;
        for (int s = s_beg; s < s_end; s++) {
            // pass 1: block length 4096, butterfly j = t over positions t + 512 q
            {
                P2 v[8];
                if (dbg_ok(s < p.sc && (x + 1) * 4096 <= p.N, kDbgScratch | kDbgTile)) {
                    const float4 *zr = reinterpret_cast<const float4 *>(p.Z) + (size_t)s * p.N + (size_t)x * 4096;
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        const float4 e = ld_no_l1(zr + t + 512 * q);  // read once
                        v[q] = ZSPLIT ? make_p2(e.x, e.y, e.z, e.w) : P2{make_float2(e.x, e.y), make_float2(e.z, e.w)};
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 8; q++) v[q] = P2{};
                }
                Dft<8>::run(v);
                const float2 *tw = p.twB + p.pass[0].off + t * 7;
#pragma unroll
                for (int q = 1; q < 8; q++) v[q] = cmul(v[q], __ldg(tw + q - 1));
#pragma unroll
                for (int q = 0; q < 8; q++) row[pad8(t + 512 * q)] = v[q];
            }
            __syncthreads();
            // passes 2 and 3: block length 512 (b = t / 64, j = t % 64) and 64 (b = t / 8, j = t % 8)
#pragma unroll
            for (int k = 1; k < 3; k++) {
                const int m = k == 1 ? 64 : 8;
                const int j = t & (m - 1), bbase = (t / m) * (8 * m) + j;
                P2 v[8];
#pragma unroll
                for (int q = 0; q < 8; q++) v[q] = row[pad8(bbase + m * q)];
                Dft<8>::run(v);
                const float2 *tw = p.twB + p.pass[k].off + j * 7;
#pragma unroll
                for (int q = 1; q < 8; q++) v[q] = cmul(v[q], __ldg(tw + q - 1));
#pragma unroll
                for (int q = 0; q < 8; q++) row[pad8(bbase + m * q)] = v[q];
                __syncthreads();
            }
            // pass 4: block length 8, outputs 8t .. 8t+7: detection and accumulation
            {
                P2 v[8];
#pragma unroll
                for (int q = 0; q < 8; q++) v[q] = row[pad8(8 * t + q)];
                Dft<8>::run(v);
#pragma unroll
                for (int q = 0; q < 8; q++) acc_add<2>(acc[q], v[q]);
            }
            // end of a register run with more spectra to come: into the slot
            if (((s - s_beg) % kRow2048Run) == kRow2048Run - 1 && s + 1 < s_end) {
                flush(first);
                first = false;
#pragma unroll
                for (int q = 0; q < 8; q++) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            __syncthreads();  // the row is free for the next spectrum
        }
        flush(first);
    }
}

// ------------------------------------------------------------ sub-bands --
// Eight-sub-band modes (16 FFTs in parallel, §4): the input interleaves nsub
// sub-bands per time sample, [time][sub][pol][re, im]. This kernel copies a
// run of M time samples of every sub-band into sub-band-contiguous slots,
// out[b * slot + m] = in[m * nsub + b], through a shared-memory tile so that
// both sides are coalesced. W is one sample of every polarisation (4 bytes
// dual-pol, 2 bytes single-pol).
template <typename W>
__global__ void deinterleave_kernel(const W *in, W *out, int nsub, long long M, long long slot) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    W *tile = reinterpret_cast<W *>(smem_raw);  // [256][nsub + 1]
    const long long m0 = (long long)blockIdx.x * 256;
    const int cnt = (int)min(256LL, M - m0);
    const int ld = nsub + 1;
    for (int e = threadIdx.x; e < cnt * nsub; e += blockDim.x) {
        const int m = e / nsub, b = e - m * nsub;
        tile[m * ld + b] = in[(m0 + m) * nsub + b];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * nsub; e += blockDim.x) {
        const int b = e / cnt, m = e - b * cnt;
        out[(long long)b * slot + m0 + m] = tile[m * ld + b];
    }
}

// ------------------------------------------------------------------ reduce --
// First level of the fold when there are many slots (small transforms split
// over many CTAs): slot group g (slots 16g .. 16g+15) is summed, in slot
// order, into slot 16g; the compensated variant sums the compensated values
// with Kahan additions and leaves a zero compensation. blockDim (32, 8):
// 32 positions x 8 slot lanes; gridDim (ceil(N / 32), groups of 16).
template <int NPOL, bool KAHAN>
__global__ void __launch_bounds__(256) fold_slots_kernel(void *partial, void *partial_comp, int slots, int N) {
    using A = typename Elem<NPOL>::Acc;
    __shared__ A lane_sum[8][32];
    __shared__ A lane_comp[8][32];
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int y = threadIdx.y;
    const int g0 = blockIdx.y * 16;
    A *pp = reinterpret_cast<A *>(partial);
    A *pc = reinterpret_cast<A *>(partial_comp);
    A s, c;
    if constexpr (NPOL == 2) s = make_float4(0.f, 0.f, 0.f, 0.f);
    else s = 0.f;
    c = s;
    if (i < N) {
        for (int g = g0 + y; g < min(slots, g0 + 16); g += 8) {
            const size_t o = (size_t)g * N + i;
            if constexpr (KAHAN) {
                if constexpr (NPOL == 2) kahan_add(s, c, sub4(pp[o], pc[o]));
                else kahan_add(s, c, pp[o] - pc[o]);
            } else if constexpr (NPOL == 2) {
                const float4 v = pp[o];
                s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
            } else {
                s += pp[o];
            }
        }
    }
    lane_sum[y][threadIdx.x] = s;
    lane_comp[y][threadIdx.x] = c;
    __syncthreads();  // every lane has read its slots before slot g0 is written
    if (y != 0 || i >= N) return;
    if constexpr (KAHAN) {
        A t, tc;
        if constexpr (NPOL == 2) {
            t = sub4(s, c);
            tc = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            t = s - c;
            tc = 0.f;
        }
#pragma unroll
        for (int l = 1; l < 8; l++) {
            if constexpr (NPOL == 2) kahan_add(t, tc, sub4(lane_sum[l][threadIdx.x], lane_comp[l][threadIdx.x]));
            else kahan_add(t, tc, lane_sum[l][threadIdx.x] - lane_comp[l][threadIdx.x]);
        }
        if constexpr (NPOL == 2) {
            pp[(size_t)g0 * N + i] = sub4(t, tc);
            pc[(size_t)g0 * N + i] = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            pp[(size_t)g0 * N + i] = t - tc;
            pc[(size_t)g0 * N + i] = 0.f;
        }
    } else {
#pragma unroll
        for (int l = 1; l < 8; l++) {
            const A v = lane_sum[l][threadIdx.x];
            if constexpr (NPOL == 2) {
                s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
            } else {
                s += v;
            }
        }
        pp[(size_t)g0 * N + i] = s;
    }
}

// The same fold for 2048-point rows (row passes radix 16, 16, 8), N2 >= 16,
// through a shared-memory tile so that both the slot reads and the
// accumulator writes are coalesced. Row position posB = 128 q1 + 8 q2 + q3
// holds k1 = q1 + 16 q2 + 256 q3, so the PB positions 128 q1 + PB g ..
// + PB - 1 (PB / 8 values of q2, all q3) are contiguous in a slot row and,
// for each of them, 16 consecutive k2 are 16 consecutive channels. A block
// takes 16 consecutive k2 (16 scattered rows pos = invA[k2]) x those PB
// positions. Lane l of L sums slots l, l + L, ... of each element into its
// tile; the lanes' tiles are then added in order and the result into
// d_accum. Grid: N2 / 16 x 16 x (128 / PB) blocks of 16 PB L threads (at
// most 512: PB = 32 runs two elements per thread); the short form, with more
// CTAs and lanes, is for small N2 with many slots.
template <int NPOL, int PB, int L>
__global__ void __launch_bounds__(512) reduce2048_kernel(const void *partial, int groups, int stride, int N,
                                                         int N2, const int *invA, void *out) {
    using A = typename Elem<NPOL>::Acc;
    constexpr int Q2G = PB / 8;  // q2 values per block
    constexpr int E = 16 * PB;   // tile elements
    __shared__ A tile[L][16][PB + 1];  // [lane][k2 offset][position offset], one pad column
    const int nk = N2 / 16;
    const int k2_0 = 16 * (blockIdx.x % nk);
    const int q1 = (blockIdx.x / nk) % 16, g = blockIdx.x / (nk * 16);
    const int p0 = 128 * q1 + PB * g;
    const A *pp = reinterpret_cast<const A *>(partial);
    for (int e = threadIdx.x; e < E * L; e += blockDim.x) {
        const int l = e / E, r = (e % E) / PB, j = e % PB;
        const size_t idx = (size_t)__ldg(invA + k2_0 + r) * 2048 + p0 + j;
        A s;
        if constexpr (NPOL == 2) s = make_float4(0.f, 0.f, 0.f, 0.f);
        else s = 0.f;
        for (int gs = l; gs < groups; gs += L) {
            const A v = pp[(size_t)gs * stride * N + idx];
            if constexpr (NPOL == 2) {
                s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
            } else {
                s += v;
            }
        }
        tile[l][r][j] = s;
    }
    __syncthreads();
    A *o = reinterpret_cast<A *>(out);
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const int r = e & 15, j = e >> 4;  // position offset j = 8 (q2 - Q2G g) + q3
        const int k1 = q1 + 16 * (Q2G * g + (j >> 3)) + 256 * (j & 7);
        const size_t k = (size_t)k1 * N2 + k2_0 + r;
        A v = tile[0][r][j];
#pragma unroll
        for (int l = 1; l < L; l++) {
            const A w = tile[l][r][j];
            if constexpr (NPOL == 2) {
                v.x += w.x; v.y += w.y; v.z += w.z; v.w += w.w;
            } else {
                v += w;
            }
        }
        if constexpr (NPOL == 2) {
            const float4 a = o[k];
            o[k] = make_float4(a.x + v.x, a.y + v.y, a.z + v.z, a.w + v.w);
        } else {
            o[k] += v;
        }
    }
}

// Fold of the partial-sum slots into the caller's accumulator, with the
// digit-reversal scatter of the four-step FFT: channel k = k1 * N2 + k2 sits
// at position invA[k2] * N1 + invB[k1] of every slot (slot g at g * stride).
// A block is 32 channels x 8 slot lanes (blockDim (32, 8)): lane y sums
// slots y, y + 8, ..., and lane 0 adds the eight lane sums in order.
template <int NPOL>
__global__ void __launch_bounds__(256) reduce_kernel(const void *partial, int groups, int stride, int N, int N1,
                                                     int N2, const int *invA, const int *invB, void *out) {
    using A = typename Elem<NPOL>::Acc;
    __shared__ A lane_sum[8][32];
    const int k = blockIdx.x * 32 + threadIdx.x;
    const int y = threadIdx.y;
    const A *pp = reinterpret_cast<const A *>(partial);
    A s;
    if constexpr (NPOL == 2) s = make_float4(0.f, 0.f, 0.f, 0.f);
    else s = 0.f;
    size_t idx = 0;
    if (k < N) {
        const int k2 = k & (N2 - 1), k1 = k / N2;
        idx = (size_t)__ldg(invA + k2) * N1 + __ldg(invB + k1);
        for (int g = y; g < groups; g += 8) {
            const A v = pp[(size_t)g * stride * N + idx];
            if constexpr (NPOL == 2) {
                s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
            } else {
                s += v;
            }
        }
    }
    lane_sum[y][threadIdx.x] = s;
    __syncthreads();
    if (y != 0 || k >= N) return;
    A *o = reinterpret_cast<A *>(out);
#pragma unroll
    for (int l = 1; l < 8; l++) {
        const A v = lane_sum[l][threadIdx.x];
        if constexpr (NPOL == 2) {
            s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
        } else {
            s += v;
        }
    }
    if constexpr (NPOL == 2) {
        const float4 a = o[k];
        o[k] = make_float4(a.x + s.x, a.y + s.y, a.z + s.z, a.w + s.w);
    } else {
        o[k] += s;
    }
}

// Compensated fold: each lane keeps a Kahan sum of its slots' compensated
// partials; lane 0 folds the eight lanes' compensated totals with Kahan
// additions and then adds the result into the caller's accumulator with the
// plan-owned compensation out_comp (cleared by vspec_dump).
template <int NPOL>
__global__ void __launch_bounds__(256) reduce_kahan_kernel(const void *partial, const void *partial_comp,
                                                           int groups, int stride, int N, int N1, int N2,
                                                           const int *invA, const int *invB, void *out,
                                                           void *out_comp) {
    using A = typename Elem<NPOL>::Acc;
    __shared__ A lane_sum[8][32];
    const int k = blockIdx.x * 32 + threadIdx.x;
    const int y = threadIdx.y;
    const A *pp = reinterpret_cast<const A *>(partial);
    const A *pc = reinterpret_cast<const A *>(partial_comp);
    A s, c;
    if constexpr (NPOL == 2) s = make_float4(0.f, 0.f, 0.f, 0.f);
    else s = 0.f;
    c = s;
    if (k < N) {
        const int k2 = k & (N2 - 1), k1 = k / N2;
        const size_t idx = (size_t)__ldg(invA + k2) * N1 + __ldg(invB + k1);
        for (int g = y; g < groups; g += 8) {
            const size_t o = (size_t)g * stride * N + idx;
            if constexpr (NPOL == 2) kahan_add(s, c, sub4(pp[o], pc[o]));
            else kahan_add(s, c, pp[o] - pc[o]);
        }
    }
    if constexpr (NPOL == 2) lane_sum[y][threadIdx.x] = sub4(s, c);
    else lane_sum[y][threadIdx.x] = s - c;
    __syncthreads();
    if (y != 0 || k >= N) return;
    A t = lane_sum[0][threadIdx.x], tc;
    if constexpr (NPOL == 2) tc = make_float4(0.f, 0.f, 0.f, 0.f);
    else tc = 0.f;
#pragma unroll
    for (int l = 1; l < 8; l++) kahan_add(t, tc, lane_sum[l][threadIdx.x]);
    A *o = reinterpret_cast<A *>(out);
    A *oc = reinterpret_cast<A *>(out_comp);
    A a = o[k], ac = oc[k];
    if constexpr (NPOL == 2) kahan_add(a, ac, sub4(t, tc));
    else kahan_add(a, ac, t - tc);
    kahan_settle(a, ac);
    o[k] = a;
    oc[k] = ac;
}

// ------------------------------------------------------ plan-time tables ---
// All plan tables are computed in FP64 and rounded once to FP32. (Defined in
// one translation unit: the others define VSPEC_NO_PLAN_TABLES.)
#ifndef VSPEC_NO_PLAN_TABLES

constexpr double kPi = 3.14159265358979323846;

// W_L^m = exp(-2 pi i m / L) for 0 <= m < L.
__device__ __forceinline__ float2 root_of_unity(long long m, long long L) {
    const double a = 2.0 * (double)m / (double)L;
    double s, c;
    sincospi(a, &s, &c);
    return make_float2((float)c, (float)-s);
}

// Pre-filter coefficients, h[i] = w[i] * sinc((i - (L-1)/2) / N) (PFB) or w[i]
// (direct), with the symmetric window w of length L.
__global__ void gen_coef_kernel(float *h, int N, int L, int pfb, int window) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L) return;
    double w = 1.0;
    if (window != 0 && L > 1) {
        const double c = cospi(2.0 * (double)i / (double)(L - 1));
        w = (window == 1) ? 0.5 - 0.5 * c : 0.54 - 0.46 * c;
    }
    double v = w;
    if (pfb) {
        const double u = ((double)i - 0.5 * (double)(L - 1)) / (double)N;
        v = (u == 0.0) ? w : w * sinpi(u) / (kPi * u);
    }
    h[i] = (float)v;
}

// Twiddles of one DIF pass: tw[off + j*(r-1) + q-1] = W_lb^(j*q).
__global__ void gen_pass_tw_kernel(float2 *tw, Pass ps) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = ps.m * (ps.r - 1);
    if (e >= n) return;
    const int j = e / (ps.r - 1), q = e - j * (ps.r - 1) + 1;
    tw[ps.off + e] = root_of_unity((long long)j * q, ps.lb);
}

// Four-step twiddles in pass-output row order: twZ[pos][n1] = W_N^(n1 * k2(pos)).
__global__ void gen_twz_kernel(float2 *twZ, int N, int N1, int N2, const int *digrevA) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)N) return;
    const int pos = (int)(e / N1), n1 = (int)(e - (long long)pos * N1);
    const long long m = ((long long)n1 * digrevA[pos]) % N;
    twZ[e] = root_of_unity(m, N);
}
#endif  // VSPEC_NO_PLAN_TABLES

}  // namespace vspec
