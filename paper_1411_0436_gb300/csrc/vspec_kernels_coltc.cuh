// vspec_kernels_coltc.cuh — kernel A with the column DFTs on the tensor cores.
//
// Same work as fir_colreg_kernel (§4: pre-filter, then the length-N2 column
// DFTs of the four-step FFT, times W_N^(n1 k2), into the chunk scratch), for
// dual-pol PFB plans of 5 to 8 taps with N2 = 16, 32 or 64 (512-point column
// tiles, C = 512 / N2 columns). The FIR runs on the CUDA cores from the same
// register window as fir_colreg_kernel. The column DFTs of a batch of SPB
// spectra are then one dense real matrix product per 128 rows:
//
//   D (rows x 2 N2) = Y (rows x 2 N2) . F (2 N2 x 2 N2),
//   row = 8 (2 (u C/8 + c/8) + p) + c % 8  (spectrum u, polarisation p, column c:
//   the two polarisations of 8 columns in consecutive 8-row groups),
//   K index 2 n2 + {0: re, 1: im},  N index 2 k2 + {0: re, 1: im},
//   F[2n2][2k2] = cos, F[2n2][2k2+1] = -sin, F[2n2+1][2k2] = sin,
//   F[2n2+1][2k2+1] = cos  of 2 pi n2 k2 / N2,
//
// so D's row holds sum_n2 y[n1 + N1 n2] W_N2^(n2 k2) in natural k2 order
// (times a power of two, kColTc*, that keeps the fp16 low parts normal).
// Y has two buffers in shared memory and D two in tensor memory: while the
// tensor cores compute batch b, the CUDA cores run the epilogue of batch
// b - 1 and then pre-filter batch b + 1 into the other Y buffer, so the
// products are off the critical path.
// Y and F are split into fp16 high and low parts (x = hi + lo, hi =
// fp16(x), lo = fp16(x - hi)) and three tcgen05.mma terms, Y_hi F_hi +
// Y_lo F_hi + Y_hi F_lo, accumulate in FP32 in tensor memory: about 22
// significant bits of each operand (the dropped Y_lo F_lo is below 2^-22).
// The two small terms are issued first and the large Y_hi F_hi last: the
// tensor cores' FP32 accumulation loses low bits relative to the running
// sum, so the small terms are summed while it is still small, and only the
// last K / 16 steps add at full magnitude.
// Both low parts matter: an emulation of this stage with Y rounded to fp16
// alone gives 9e-4 of the spectrum RMS on a one-spectrum dump of the
// 131072-channel workload, with F rounded to fp16 hi + lo alone 4e-6.
// FIR outputs stay below 2^9 in magnitude and the DFT coefficients below 1,
// well inside fp16's range. One thread issues the MMAs; tcgen05.commit
// signals an mbarrier that the CTA waits on with a bounded spin (status word
// and a clean exit if it gives up). The epilogue reads D with the .16x256b
// shape of tcgen05.ld, which gives each thread two adjacent columns (re, im
// of one output) of two rows 8 apart: by the row order above, the X and Y
// polarisations of the same output. It multiplies them by W_N^(n1 k2) (a copy
// of the four-step twiddles scaled by 2^-12, loaded once per tile into free
// columns of the thread's own tensor-memory lane and read back beside D; the
// tile's coefficients stay in registers: shared memory holds only the
// operands and the staged frames) and writes whole 16-byte scratch elements
// (X.re, X.im, Y.re, Y.im), the order in which the 2048-point row kernel
// reads them (its ZSPLIT form).
//
// Shared-memory operands (K-major, no swizzle): 8-row x 16-byte core
// matrices, element (row r, k) at byte
//   (r / 8) * SBO + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,  SBO = 2 N2 * 16,
// so the K step between core matrices is 128 bytes and one K = 16 slice of
// an MMA is 256 bytes further on. The row order above, with the thread order
// of ColTc::pt_*, puts the eight columns a warp's threads stage for one
// spectrum and polarisation in eight different rows of one core matrix: the
// stores are free of bank conflicts.
#pragma once
#include <cuda_fp16.h>

#include "vspec_kernels.cuh"
#include "vspec_tc.cuh"

namespace vspec {

// Power-of-two scaling of the operands, exact in both directions: the FIR
// coefficients are scaled by 2^4 and F by 2^8, so that the low fp16 parts of
// small values stay normal numbers (above 2^-14), and the four-step twiddles
// by 2^-12 to undo both.
constexpr float kColTcYScale = 16.0f;
constexpr double kColTcFScale = 256.0;
constexpr float kColTcUnscale = 1.0f / 4096.0f;

template <int N2>
struct ColTc {
    static constexpr int PT = 8, PTS = 512, C = PTS / N2, SPB = 8;
    static constexpr int K = 2 * N2, NN = 2 * N2;  // MMA K and N
    static constexpr int ROWS = SPB * 2 * C;       // rows of Y: (spectrum, polarisation, column)
    static constexpr int MB = ROWS / 128;          // M = 128 blocks
    static constexpr int SBO = K * 16;             // bytes between 8-row groups
    static constexpr int APART = ROWS * K * 2;     // bytes of one fp16 part of Y
    static constexpr int BPART = NN * K * 2;       // bytes of one fp16 part of F
    static constexpr int KSTEPS = K / 16;
    static constexpr int TMEM_COLS = MB * NN;      // fp32 columns of one D buffer
    // tensor memory: D buffers 0 and 1, then each epilogue thread's 16
    // twiddles (32 columns per thread column group g, 4 groups)
    static constexpr int TMEM_ALLOC = 4 * TMEM_COLS;
    // two A buffers (Y hi, Y lo), F hi, F lo, raw frames [2][SPB][PTS] u32
    static constexpr size_t smem = 4 * (size_t)APART + 2 * (size_t)BPART + 2 * (size_t)SPB * PTS * 4;
    static_assert(N2 == 16 || N2 == 32 || N2 == 64, "column lengths of this kernel");
    static_assert(C % 8 == 0 && SPB % 4 == 0 && PTS % 4 == 0, "whole core-matrix row groups, whole copy rounds");
    static_assert(MB * 128 == ROWS && TMEM_COLS == 128, "2 accumulators of 128 TMEM columns, whole M blocks");
    static_assert(2 * TMEM_COLS + 4 * 32 <= TMEM_ALLOC, "twiddle columns after the accumulators");
    // Thread t pre-filters point (n2, c) of the tile, laid out so that every
    // warp holds 8 consecutive columns x 4 consecutive n2: its stores of Y
    // then fill 8 rows x 4 words of one core matrix, free of bank conflicts.
    // The staged frames use the same order (4 consecutive columns stay
    // adjacent, one 16-byte copy).
    static constexpr int CB = C / 8;
    __host__ __device__ static constexpr int pt_n2(int t) { return ((t >> 5) / CB) * 4 + ((t >> 3) & 3); }
    __host__ __device__ static constexpr int pt_c(int t) { return ((t >> 5) % CB) * 8 + (t & 7); }
    __host__ __device__ static constexpr int pt_index(int n2, int c) {
        return ((n2 >> 2) * CB + (c >> 3)) * 32 + (n2 & 3) * 8 + (c & 7);
    }
    static_assert(smem <= 232448 - 1024, "shared memory of one CTA");
    __host__ __device__ static constexpr int off(int r, int k) {
        return (r >> 3) * SBO + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
    }
};

// The column DFT operand F of ColTc<N2> as its shared-memory image, hi part
// then lo part (from FP64 cosines and sines, rounded once to fp16 each).
__global__ void gen_coltc_operand_kernel(unsigned char *op, int N2) {
    const int NN = 2 * N2, K = 2 * N2;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NN * K) return;
    const int n = e / K, k = e % K;            // D column (output), K index (input)
    const int k2 = n >> 1, n2 = k >> 1;
    double sn, cs;
    sincospi(2.0 * (double)((n2 * k2) % N2) / (double)N2, &sn, &cs);
    // (xr + i xi)(cos - i sin): re gets xr cos + xi sin, im gets -xr sin + xi cos
    double v;
    if ((n & 1) == 0) v = (k & 1) ? sn : cs;
    else v = (k & 1) ? cs : -sn;
    v *= kColTcFScale;
    const __half hi = __double2half(v);
    const __half lo = __double2half(v - (double)__half2float(hi));
    const int SBO = K * 16;
    const int o = (n >> 3) * SBO + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
    *reinterpret_cast<__half *>(op + o) = hi;
    *reinterpret_cast<__half *>(op + NN * K * 2 + o) = lo;
}

// The four-step twiddles W_N^(n1 k2) times 2^-12 (exact) for the epilogue of
// fir_coltc_kernel, stored after F in the plan's operand array, tile by tile:
// entry x * 512 + k2 * C + c is column n1 = x * C + c of tile x (C = 512 /
// N2), so that a tile's twiddles are one contiguous 4 KiB block in L1.
__global__ void gen_coltc_twz_kernel(float2 *dst, const float2 *twZ, int N, int N1, int N2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    const int C = 512 / N2, x = e / 512, r = e % 512, k2 = r / C, c = r % C;
    const float2 w = twZ[(size_t)k2 * N1 + x * C + c];
    dst[e] = make_float2(w.x * kColTcUnscale, w.y * kColTcUnscale);
}

// The chunk-scratch stores of the epilogue (64 KiB per batch, never read
// back by this kernel) do not allocate in L1.
__device__ __forceinline__ void st_no_l1(float4 *ptr, float4 v) {
    asm volatile("st.global.L1::no_allocate.v4.f32 [%0], {%1, %2, %3, %4};"
                 :: "l"(ptr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
}

// hi/lo fp16 split of both polarisations of a complex value, y = (re, im)
// with re = (X.re, Y.re), im = (X.im, Y.im), into packed half2 words (re,
// im) per polarisation. The high part is y with its mantissa truncated to
// fp16's 11 significant bits (exact in fp16 for the operands' range), so the
// low part y - hi is exact in FP32 and then rounds once to fp16: |lo| <
// 2^-10 |y|, hi + lo within 2^-21 |y| of y. On the packed pairs this takes
// four bit masks, two paired subtractions and four conversions.
__device__ __forceinline__ void split_p2(const P2 &y, uint32_t &hx, uint32_t &lx, uint32_t &hy, uint32_t &ly) {
    constexpr unsigned kMask = 0xFFFFE000u;
    const float2 hr = make_float2(__uint_as_float(__float_as_uint(y.re.x) & kMask),
                                  __uint_as_float(__float_as_uint(y.re.y) & kMask));
    const float2 hi = make_float2(__uint_as_float(__float_as_uint(y.im.x) & kMask),
                                  __uint_as_float(__float_as_uint(y.im.y) & kMask));
    const float2 lr = sub2(y.re, hr), li = sub2(y.im, hi);
    const __half2 a = __floats2half2_rn(hr.x, hi.x), b = __floats2half2_rn(hr.y, hi.y);
    const __half2 c = __floats2half2_rn(lr.x, li.x), d = __floats2half2_rn(lr.y, li.y);
    hx = *reinterpret_cast<const uint32_t *>(&a);
    hy = *reinterpret_cast<const uint32_t *>(&b);
    lx = *reinterpret_cast<const uint32_t *>(&c);
    ly = *reinterpret_cast<const uint32_t *>(&d);
}

// fp16 instruction descriptor of kind::f16: fp32 D (bits 4-5 = 1), fp16 A and
// B (type 0), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t instr_desc_f16(int m, int n) {
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

template <int N2>
__global__ void __launch_bounds__(512, 1) fir_coltc_kernel(const __grid_constant__ ColParams p) {
    using G = ColTc<N2>;
    using namespace tc;
    constexpr int PT = G::PT, PTS = G::PTS, C = G::C, SPB = G::SPB;
    // the plan uses this kernel only with 2048-point rows: the transform
    // length and row stride are compile-time constants (immediate offsets)
    constexpr int N1 = 2048;
    constexpr long long NCH = (long long)N1 * N2;
    extern __shared__ __align__(128) unsigned char smem_ct[];
    // A buffer b: hi part at smem_ct + 2 b APART, lo part APART further on
    unsigned char *fhi = smem_ct + 4 * G::APART, *flo = fhi + G::BPART;
    uint32_t *raw = reinterpret_cast<uint32_t *>(flo + G::BPART);  // [2][SPB][PTS]
    // W_N^(n1 k2) * 2^-12 in natural k2 order, [tile][k2][c] (after F in the operand array)
    const float2 *twsc = reinterpret_cast<const float2 *>(p.dftop + 2 * G::BPART);
    __shared__ __align__(8) uint64_t mbar[2];  // MMA completion of the batches in D buffer 0 / 1
    __shared__ uint32_t tmem_slot;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int D = PT - p.P;  // leading zero taps

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_addr(&tmem_slot)), "r"((uint32_t)G::TMEM_ALLOC) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // F (hi and lo) into shared memory, 16 bytes at a time
    for (int e = t; e < 2 * G::BPART / 16; e += blockDim.x)
        reinterpret_cast<uint4 *>(fhi)[e] = __ldg(reinterpret_cast<const uint4 *>(p.dftop) + e);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    // F's descriptors (fixed for the kernel)
    const uint64_t dfhi = smem_desc(smem_addr(fhi), 128u, G::SBO), dflo = smem_desc(smem_addr(flo), 128u, G::SBO);
    static_assert(G::smem + 1024 < (1u << 18), "descriptor start addresses: 14 bits of address / 16");

    // The epilogue's share of D: lane quarter q of TMEM, the 32 columns from
    // 32 g (M block mb, outputs k2 = k0 .. k0 + 15), read as two 16-lane
    // halves h. Half h holds the 8-row groups 16 mb + 4 q + 2 h (X) and + 1
    // (Y) of spectrum eu[h], columns 8 ecb[h] .. 8 ecb[h] + 7; this thread
    // gets column ec[h] = 8 ecb[h] + lane / 4 and outputs k2 = k0 + 4 r + lane % 4.
    const int q = warp & 3, g = warp >> 2;
    const int mb = (32 * g) / G::NN, k0 = ((32 * g) % G::NN) / 2;
    int eu[2], ec[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int pr = 8 * mb + 2 * q + h;  // (u C/8 + c/8) of the half's groups
        eu[h] = pr / (C / 8);
        ec[h] = (pr % (C / 8)) * 8 + (lane >> 2);
    }
    const int n2 = G::pt_n2(t), c = G::pt_c(t);  // the point this thread pre-filters
    // its operand offsets for spectrum u of a batch: o_y + 2 u (C / 8) SBO (X)
    // and one 8-row group further (Y), C a multiple of 8
    const int o_y = G::off(16 * (c >> 3) + (c & 7), 2 * n2);
    // its share of the frame staging: 16-byte copies e = t + PTS i, i < SPB / 4,
    // of frame u = t / (PTS / 4) + 4 i, tile row rn2, columns 4 ch .. 4 ch + 3
    constexpr int per_row = C / 4, per_frame = PTS / 4;
    const int st_u = t / per_frame, st_r = t % per_frame, st_n2 = st_r / per_row, st_ch = st_r % per_row;
    const int st_dst = st_u * PTS + G::pt_index(st_n2, st_ch * 4);

    bool ok = true;
    // Batch gi (counted over the CTA's tiles) uses A buffer and D buffer gi & 1
    // and is the (gi >> 1)-th commit on mbar[gi & 1]. Batch gi - 2 is waited
    // for before batch gi writes its A buffer, so the waits on each mbarrier
    // alternate with its commits and the phase parity is never ambiguous.
    uint32_t gi = 0;
    const TileSplit sp = tile_split(p.tiles, p.sc, p.G);
    for (long long f = sp.lo; f < sp.hi && ok;) {
        const long long base = f / p.sc * p.sc;  // first item of this super-tile
        const int x = (int)(f / p.sc) * sp.G + sp.r;
        const int s_beg = (int)(f - base);
        const int s_end = (int)(min(sp.hi, base + p.sc) - base);
        f = base + s_end;
        const int n1_0 = x * C;
        const long long n_pt = n1_0 + c + (long long)N1 * n2;
        // this point's coefficients (times 2^4), kept in registers for the tile
        float2 cf2[PT];
#pragma unroll
        for (int k = 0; k < PT; k++)
            cf2[k] = dup2(k >= D ? __ldg(p.coef + (size_t)(k - D) * NCH + n_pt) * kColTcYScale : 0.f);
        P2 win[PT];
        const long long sabs = p.s0 + s_beg;
#pragma unroll
        for (int k = 0; k < PT - 1; k++) {
            long long fr = sabs - D + k;
            if (fr < 0) fr = 0;
            win[k] = unpack_p2(load_raw<2>(p.in, fr * NCH + n_pt) ^ 0x80808080u);
        }
        // this thread's epilogue twiddles W_N^(n1 k2) 2^-12 (column ec[h],
        // k2 = k0 + 4 r + lane % 4) into its TMEM lane (the previous tile's
        // epilogues are done with them: the barrier that ended that tile)
        const uint32_t ttw = tmem + ((uint32_t)(32 * q) << 16) + 2u * G::TMEM_COLS + (uint32_t)(32 * g);
        {
            float w[16];
#pragma unroll
            for (int h = 0; h < 2; h++)
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const float2 v = __ldg(twsc + (size_t)x * PTS + (k0 + 4 * r + (lane & 3)) * C + ec[h]);
                    w[8 * h + 2 * r] = v.x;
                    w[8 * h + 2 * r + 1] = v.y;
                }
            tmem_st16_wait(ttw, w);
        }
        // frames of the tile, from spectrum 0 of the chunk on (newest frame
        // of each spectrum: P - 1 frames after the spectrum's first)
        const uint32_t *st_src = reinterpret_cast<const uint32_t *>(p.in) + (p.s0 + st_u + p.P - 1) * NCH + n1_0 +
                                 (long long)N1 * st_n2 + st_ch * 4;
        auto stage = [&](int sb, int buf) {
            const int nbb = min(SPB, s_end - sb);
            const uint32_t *src = st_src + (long long)sb * NCH;
            const uint32_t dst = (uint32_t)__cvta_generic_to_shared(raw + buf * SPB * PTS + st_dst);
#pragma unroll
            for (int i = 0; i < SPB / 4; i++)
                if (st_u + 4 * i < nbb)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                                 :: "r"(dst + 16u * PTS * i), "l"(src + 4 * i * NCH) : "memory");
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        // Wait for batch bi's MMAs (warp-uniform answer), then its epilogue:
        // from D buffer bi & 1, per half h, both polarisations of outputs
        // k2 = k0 + 4 r + lane % 4 (r < 4) of column ec[h], spectrum eu[h] of
        // the batch, times W_N^(n1 k2), into the scratch as whole elements.
        // tcgen05.ld is warp-collective: every lane loads, lanes past the
        // batch's spectra skip the stores.
        auto finish = [&](int sbase, int nbb, uint32_t bi) {
            bool done = mbar_wait(&mbar[bi & 1u], (bi >> 1) & 1u, p.wait_limit);
            done = __all_sync(0xffffffffu, done);
            if (done) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const uint32_t ta = tmem + ((uint32_t)(32 * q + 16 * h) << 16) + (bi & 1u) * G::TMEM_COLS +
                                        (uint32_t)(32 * g);
                    float d[16], w[8];  // 4 outputs of both polarisations, their twiddles
                    tmem_ld_pairs(ta, ttw + 8u * h, d, w);
                    if (eu[h] < nbb) {
                        float4 *z = reinterpret_cast<float4 *>(p.Z) + (size_t)(sbase + eu[h]) * NCH + n1_0 + ec[h];
#pragma unroll
                        for (int r = 0; r < 4; r++) {
                            const int k2 = k0 + 4 * r + (lane & 3);
                            const float2 tw = make_float2(w[2 * r], w[2 * r + 1]);
                            const float2 xo = cmul(make_float2(d[4 * r], d[4 * r + 1]), tw);
                            const float2 yo = cmul(make_float2(d[4 * r + 2], d[4 * r + 3]), tw);
                            st_no_l1(z + (size_t)k2 * N1, make_float4(xo.x, xo.y, yo.x, yo.y));
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            return done;
        };
        int pend_base = 0, pend_nb = 0;  // the batch issued last, its epilogue pending
        stage(s_beg, 0);
        for (int s_base = s_beg, buf = 0; s_base < s_end; s_base += SPB, buf ^= 1) {
            const int nb = min(SPB, s_end - s_base);
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            // frames visible; the other frame buffer is free; the epilogue of
            // batch gi - 2 is done with D buffer gi & 1 and its MMAs with A
            // buffer gi & 1; every thread's waits so far succeeded
            ok = __syncthreads_and(ok);
            if (!ok) break;
            if (s_base + SPB < s_end) stage(s_base + SPB, buf ^ 1);
            const uint32_t ab = gi & 1u;
            unsigned char *ahi = smem_ct + 2 * ab * G::APART, *alo = ahi + G::APART;
            // FIR of spectrum u of the batch into rows (2u + p) C + c of Y, K = 2 n2
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
                uint32_t hx, lx, hy, ly;
                split_p2(y, hx, lx, hy, ly);
                constexpr int ou = 2 * u * (C / 8) * G::SBO;
                const int ox = o_y + ou, oy = o_y + ou + G::SBO;
                *reinterpret_cast<uint32_t *>(ahi + ox) = hx;
                *reinterpret_cast<uint32_t *>(alo + ox) = lx;
                *reinterpret_cast<uint32_t *>(ahi + oy) = hy;
                *reinterpret_cast<uint32_t *>(alo + oy) = ly;
            };
            if (nb == SPB) for_slots(fir_one, std::make_integer_sequence<int, SPB>{});
            else for_slots_below(fir_one, nb, std::make_integer_sequence<int, SPB>{});
            // Y is complete: make it visible to the tensor cores, then issue
            // batch gi into D buffer ab
            fence_proxy_async();
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (t == 0) {
                constexpr uint32_t idesc = instr_desc_f16(128, G::NN);
                // small terms first: Y_lo F_hi, Y_hi F_lo, then Y_hi F_hi. A
                // descriptor's start address field is the byte address / 16 and
                // shared addresses stay below 2^18, so each operand block is its
                // part's base descriptor plus a compile-time offset / 16 (this
                // thread issues while the others wait at the next barrier).
                const uint64_t dlo = smem_desc(smem_addr(alo), 128u, G::SBO);
                const uint64_t dhi = smem_desc(smem_addr(ahi), 128u, G::SBO);
                const uint64_t as[3] = {dlo, dhi, dhi};
                const uint64_t bs[3] = {dfhi, dflo, dfhi};
#pragma unroll
                for (int m = 0; m < G::MB; m++) {
                    uint32_t acc = 0;
                    const uint32_t dcol = tmem + ab * G::TMEM_COLS + (uint32_t)(m * G::NN);
#pragma unroll
                    for (int term = 0; term < 3; term++) {
#pragma unroll
                        for (int ks = 0; ks < G::KSTEPS; ks++) {
                            const uint64_t ad = as[term] + (uint64_t)((m * 16 * G::SBO + 256 * ks) >> 4);
                            const uint64_t bd = bs[term] + (uint64_t)((256 * ks) >> 4);
                            mma_bf16(dcol, ad, bd, idesc, acc);
                            acc = 1;
                        }
                    }
                }
                mma_commit(&mbar[ab]);
            }
            // the previous batch's epilogue runs while the tensor cores work
            // on this one (and this batch's while the next one is pre-filtered)
            if (pend_nb > 0) ok = finish(pend_base, pend_nb, gi - 1);
            pend_base = s_base;
            pend_nb = nb;
            gi++;
        }
        if (ok && pend_nb > 0) ok = finish(pend_base, pend_nb, gi - 1);
        ok = __syncthreads_and(ok);  // the tile's batches are done with D and A
    }
    if (!ok && t == 0) atomicExch(p.status, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        // after a wait that gave up, MMAs may be outstanding: wait with the
        // full bound for the last batch's commit (it arrives once every MMA
        // issued before it is complete) before freeing their tensor memory
        if (!ok && gi > 0) mbar_wait(&mbar[(gi - 1) & 1u], ((gi - 1) >> 1) & 1u);
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"((uint32_t)G::TMEM_ALLOC) : "memory");
    }
}

}  // namespace vspec
