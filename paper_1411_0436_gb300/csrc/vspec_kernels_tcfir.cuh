// vspec_kernels_tcfir.cuh — kernel A as tensor-core products on the int8 input.
//
// The pre-filter (§4, PFB) and the column DFTs of the four-step FFT are both
// linear in the input, so for one column n1 they are one matrix product
// over the raw samples. With N2 = 16 Q column points split by decimation in
// time, n2 = r + Q m (residue r < Q, m < 16), and the column outputs written
// k2 = k2' + 16 q (k2' < 16, q < Q):
//
//   D_r[s][k2'] = sum_t sum_m B_{n1,r,t}[k2'][m] x_{s+t}[n1 + N1 (r + Q m)],
//   B_{n1,r,t}[k2'][m] = h[t N + n1 + N1 (r + Q m)] W_16^(m k2') W_N2^(r k2') W_N^(n1 k2'),
//   Z[s][k2' + 16 q][n1] = W_N^(16 n1 q) sum_r W_Q^(r q) D_r[s][k2'],
//
// (x_f = frame f of the input, h the P-tap coefficients, tap t on frame s+t).
// D_r is a real product with K = 32 (m, re/im) and N = 32 (k2', re/im) per
// tap. The A operand is the int8 samples themselves, exact in fp16, and the
// sum over taps needs no copy per tap: the frames of one column are stored
// once as the rows of a K-major operand whose 8-row core matrices are
// contiguous (16 bytes per row, SBO = 128), so the operand of tap t is the
// same memory with its start moved down t rows (16 t bytes). Spectrum s of a
// block of 128 uses rows s .. s + P - 1: the Hankel structure of the
// filter bank, at no staging cost. B (fp16, from FP64 products rounded
// once) is computed at plan time, Q P blocks of 2 KiB per column, and where
// shared memory allows (direct mode, and PFB with 16- or 32-point columns) a
// second set with the low parts, B - fp16(B), so that two MMA terms carry
// about 22 bits of every coefficient; the 64-point PFB form keeps the high
// parts only (about 11 bits, errors that average over the transform).
// tcgen05.mma accumulates the P taps and two K slices in FP32 in tensor
// memory; the epilogue combines the Q residues (radix Q, with W_Q = -i
// multiples only) and applies the Q - 1 column twiddles.
//
// A CTA owns one column n1 for a run of spectra, in blocks of 128 spectra
// (M = 128, one TMEM lane per spectrum). Its input is Q * 16 scattered
// 4-byte samples per frame; groups of 8 CTAs take 8 adjacent columns at
// about the same time (tile_split), so every 32-byte sector comes from HBM
// once. D is double-buffered in tensor memory: the epilogue of block b - 1
// runs while the tensor cores compute block b. Bounded waits: a wait that
// gives up sets the status word and the CTA exits cleanly.
#pragma once
#include <cuda_fp16.h>

#include "vspec_kernels.cuh"
#include "vspec_tc.cuh"

namespace vspec {

template <int Q>
struct TcFir {
    static constexpr int N2 = 16 * Q;
    static constexpr int M = 128;                  // spectra per block
    static constexpr int PMAX = 8;                 // taps held by the frame operand
    static constexpr int ROWS = M + PMAX;          // frame rows (M + P - 1 used)
    static constexpr int LBO = ROWS * 16;          // bytes between K chunks of a frame operand
    static constexpr int AMAT = 4 * LBO;           // bytes of one frame operand (4 K chunks of 8 fp16)
    static constexpr int NMAT = 2 * Q;             // frame operands: (residue, polarisation)
    static constexpr int BBLK = 32 * 32 * 2;       // bytes of one B block (fp16)
    static constexpr int RS = N2 + 1;              // raw frame stride in words (bank spread)
    static constexpr int DCOLS = NMAT * 32;        // TMEM columns of one D buffer
    static constexpr int TMEM_ALLOC = 2 * DCOLS < 32 ? 32 : 2 * DCOLS;
    // A operands, B blocks (terms parts of P taps), two raw frame buffers [ROWS][RS] u32
    static constexpr size_t smem_for(int P, int terms) {
        return (size_t)NMAT * AMAT + (size_t)Q * P * terms * BBLK + 2 * (size_t)ROWS * RS * 4;
    }
    static constexpr size_t smem = (size_t)NMAT * AMAT + (size_t)Q * PMAX * BBLK + 2 * (size_t)ROWS * RS * 4;
    static_assert(Q == 1 || Q == 2 || Q == 4, "16, 32 or 64 column points");
    static_assert(smem <= 232448 - 1024, "shared memory of one CTA");
    static_assert(2 * DCOLS <= 512, "two D buffers in tensor memory");
};

// B blocks of every column: column n1 holds `terms` sets of Q P blocks; block
// (r P + t) of set h holds the 32 x 32 real form of B_{n1,r,t} (row 2 k2' +
// {re, im} of the output, K index 2 m + {re, im}), K-major in 8 x 8 core
// matrices (SBO 512, LBO 128), as fp16: set 0 the high parts, set 1 (if
// terms == 2) the low parts.
__global__ void gen_tcfir_operand_kernel(unsigned char *op, const float *coef, int N, int N1, int Q, int P,
                                         int terms) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)N1 * Q * P * 1024;
    if (e >= total) return;
    const int within = (int)(e & 1023);
    const long long blk = e >> 10;                 // (n1 Q + r) P + t
    const int t = (int)(blk % P), r = (int)((blk / P) % Q);
    const long long n1 = blk / ((long long)P * Q);
    const int row = within >> 5, k = within & 31;  // output row 2 k2' + c', K index 2 m + c
    const int k2 = row >> 1, m = k >> 1;
    const int N2 = 16 * Q;
    const long long n = n1 + (long long)N1 * (r + (long long)Q * m);
    const double h = (double)coef[(size_t)t * N + n];
    // exponent of W_N: m k2' N/16 + r k2' N/N2 + n1 k2' (mod N)
    const long long ex = ((long long)m * k2 * (N / 16) + (long long)r * k2 * (N / N2) + n1 * k2) % N;
    double sn, cs;
    sincospi(2.0 * (double)ex / (double)N, &sn, &cs);
    const double br = h * cs, bi = -h * sn;        // b = h W, W = cos - i sin
    // (xr + i xi) b: re = xr br - xi bi, im = xr bi + xi br
    double v;
    if ((row & 1) == 0) v = (k & 1) ? -bi : br;
    else v = (k & 1) ? br : bi;
    const int o = (row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
    const size_t col = (size_t)n1 * terms * Q * P * 2048;  // this column's sets
    const size_t inblk = (size_t)(r * P + t) * 2048 + o;
    const __half hi = __double2half(v);
    *reinterpret_cast<__half *>(op + col + inblk) = hi;
    if (terms == 2)
        *reinterpret_cast<__half *>(op + col + (size_t)Q * P * 2048 + inblk) = __double2half(v - (double)__half2float(hi));
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = __uint_as_float(r[i]);
}

// One input word (X.re, X.im, Y.re, Y.im as int8, already ^ 0x80808080) as
// two fp16 pairs, exactly: 0x64uu is the fp16 1024 + u, minus 1152 gives u - 128.
__device__ __forceinline__ void unpack_half2(uint32_t w, uint32_t &x, uint32_t &y) {
    const __half2 bias = __halves2half2(__ushort_as_half(0x6480), __ushort_as_half(0x6480));  // 1152
    const uint32_t xb = __byte_perm(w, 0x64646464u, 0x5140u);
    const uint32_t yb = __byte_perm(w, 0x64646464u, 0x5342u);
    const __half2 xh = __hsub2(*reinterpret_cast<const __half2 *>(&xb), bias);
    const __half2 yh = __hsub2(*reinterpret_cast<const __half2 *>(&yb), bias);
    x = *reinterpret_cast<const uint32_t *>(&xh);
    y = *reinterpret_cast<const uint32_t *>(&yh);
}

template <int Q>
__global__ void __launch_bounds__(512, 1) fir_tcfir_kernel(const __grid_constant__ ColParams p) {
    using G = TcFir<Q>;
    using namespace tc;
    constexpr int M = G::M, ROWS = G::ROWS, RS = G::RS, N2 = G::N2;
    extern __shared__ __align__(128) unsigned char smem_tf[];
    unsigned char *amat = smem_tf;                                   // [NMAT][4][ROWS] x 16 B
    unsigned char *bops = amat + G::NMAT * G::AMAT;                  // [Q][P] blocks of 2 KiB
    uint32_t *raw = reinterpret_cast<uint32_t *>(bops + (size_t)Q * p.P * p.bterms * G::BBLK);  // [2][ROWS][RS]
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ float2 colw[4];  // W_N^(16 n1 q), q < Q
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int P = p.P;
    const int nframes_max = M + P - 1;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_addr(&tmem_slot)), "r"((uint32_t)G::TMEM_ALLOC) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        mbar_init(&mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    // epilogue share: TMEM lane quarter lq (spectra 32 lq ..), k2' group kg
    // (k2' = 4 kg .. 4 kg + 3) of every operand's D
    const int lq = warp & 3, kg = warp >> 2;
    const int srow = 32 * lq + lane;  // spectrum of the block this thread writes

    bool ok = true;
    uint32_t blocks = 0;  // MMA blocks committed (mbarrier phase, TMEM buffer)
    const TileSplit sp = tile_split(p.tiles, p.sc, p.G);
    for (long long f = sp.lo; f < sp.hi && ok;) {
        const long long base = f / p.sc * p.sc;  // first item of this super-tile
        const int n1 = (int)(f / p.sc) * sp.G + sp.r;  // the column (tiles of one column)
        const int s_beg = (int)(f - base);
        const int s_end = (int)(min(sp.hi, base + p.sc) - base);
        f = base + s_end;
        // this column's B blocks (bterms x Q P x 2 KiB) and its Q - 1 output twiddles
        {
            const int nb16 = p.bterms * Q * P * G::BBLK / 16;
            const uint4 *src = reinterpret_cast<const uint4 *>(p.dftop) + (size_t)n1 * nb16;
            for (int e = t; e < nb16; e += blockDim.x)
                reinterpret_cast<uint4 *>(bops)[e] = __ldg(src + e);
            if (t < Q) colw[t] = __ldg(p.twZ + (size_t)16 * t * p.N1 + n1);
        }
        // frames [fr0, fr0 + cnt) of this column into raw buffer `buf`: 4-byte
        // copies of the Q * 16 samples n1 + N1 n2 of each frame
        auto stage = [&](long long fr0, int cnt, int buf) {
            uint32_t *dst = raw + buf * ROWS * RS;
            for (int e = t; e < cnt * N2; e += blockDim.x) {
                const int fr = e / N2, n2 = e % N2;
                const int8_t *src = p.in + ((fr0 + fr) * p.N + n1 + (long long)p.N1 * n2) * 4;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;"
                             :: "r"((uint32_t)__cvta_generic_to_shared(dst + fr * RS + n2)), "l"(src) : "memory");
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        // epilogue of a finished block: D buffer dbuf, spectra sb0 + srow
        auto epilogue = [&](int sb0, int nsp, uint32_t dbuf) {
            float d[G::NMAT][8];  // operand (r, p): 4 complex outputs k2' = 4 kg + j
#pragma unroll
            for (int mo = 0; mo < G::NMAT; mo++)
                tmem_ld8(tmem + ((uint32_t)(32 * lq) << 16) + dbuf * (uint32_t)G::DCOLS + (uint32_t)(32 * mo + 8 * kg),
                         d[mo]);
            if (srow < nsp) {
                P2 *z = reinterpret_cast<P2 *>(p.Z) + (size_t)(sb0 + srow) * p.N + n1;
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int k2 = 4 * kg + j;
                    P2 v[Q];
#pragma unroll
                    for (int r = 0; r < Q; r++)
                        v[r] = make_p2(d[2 * r][2 * j], d[2 * r][2 * j + 1], d[2 * r + 1][2 * j], d[2 * r + 1][2 * j + 1]);
                    Dft<Q>::run(v);  // v[q] = sum_r W_Q^(r q) D_r
#pragma unroll
                    for (int q = 0; q < Q; q++) {
                        const P2 o = q == 0 ? v[0] : cmul(v[q], colw[q]);
                        z[(size_t)(k2 + 16 * q) * p.N1] = o;
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        };

        int pend_s = 0, pend_n = 0;  // the block whose MMAs are done and epilogue pending
        const int nblk = (s_end - s_beg + M - 1) / M;
        stage(p.s0 + s_beg, min(nframes_max, s_end - s_beg + P - 1), 0);
        for (int b = 0; b < nblk; b++) {
            const int sb0 = s_beg + b * M;
            const int nsp = min(M, s_end - sb0);
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncthreads();  // block b's frames visible; the other raw buffer is free
            if (b + 1 < nblk)
                stage(p.s0 + sb0 + M, min(nframes_max, s_end - sb0 - M + P - 1), (b + 1) & 1);
            // frames -> fp16 operands (the previous block's MMAs are done with
            // them: their wait ended the previous iteration). Unit (row, r, j):
            // K chunk j (m = 4 j .. 4 j + 3) of residue r for both polarisations.
            {
                const uint32_t *rb = raw + (b & 1) * ROWS * RS;
                const int nrow = min(nframes_max, nsp + P - 1);
                for (int e = t; e < nrow * Q * 4; e += blockDim.x) {
                    const int row = e % nrow, rj = e / nrow, r = rj / 4, j = rj % 4;
                    uint32_t xs[4], ys[4];
#pragma unroll
                    for (int i = 0; i < 4; i++)
                        unpack_half2(rb[row * RS + r + Q * (4 * j + i)] ^ 0x80808080u, xs[i], ys[i]);
                    unsigned char *ax = amat + (2 * r) * G::AMAT + j * G::LBO + row * 16;
                    *reinterpret_cast<uint4 *>(ax) = make_uint4(xs[0], xs[1], xs[2], xs[3]);
                    *reinterpret_cast<uint4 *>(ax + G::AMAT) = make_uint4(ys[0], ys[1], ys[2], ys[3]);
                }
            }
            fence_proxy_async();
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t dbuf = blocks & 1u;
            if (t == 0) {
                constexpr uint32_t idesc = (1u << 4) | ((uint32_t)(32 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
#pragma unroll
                for (int mo = 0; mo < G::NMAT; mo++) {  // operand (r, p) = (mo / 2, mo % 2)
                    const uint32_t a0 = smem_addr(amat + mo * G::AMAT);
                    const uint32_t b0 = smem_addr(bops + (size_t)(mo >> 1) * P * G::BBLK);
                    const uint32_t dcol = tmem + dbuf * (uint32_t)G::DCOLS + (uint32_t)(32 * mo);
                    for (int h = 0; h < p.bterms; h++) {  // the high parts, then the low parts
                        const uint32_t bh = b0 + (uint32_t)(h * Q * P * G::BBLK);
                        for (int tap = 0; tap < P; tap++) {
#pragma unroll
                            for (int ks = 0; ks < 2; ks++) {
                                const uint64_t ad = smem_desc(a0 + 16u * tap + 2u * ks * G::LBO, G::LBO, 128u);
                                const uint64_t bd = smem_desc(bh + tap * G::BBLK + 256u * ks, 128u, 512u);
                                mma_bf16(dcol, ad, bd, idesc, (h | tap | ks) ? 1u : 0u);
                            }
                        }
                    }
                }
                mma_commit(&mbar);
            }
            // the previous block's epilogue runs while the tensor cores work
            if (pend_n > 0) epilogue(pend_s, pend_n, dbuf ^ 1u);
            const bool done = mbar_wait(&mbar, dbuf, p.wait_limit);
            blocks++;
            ok = __syncthreads_and(done);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!ok) break;
            pend_s = sb0;
            pend_n = nsp;
        }
        if (ok && pend_n > 0) epilogue(pend_s, pend_n, (blocks - 1) & 1u);
        __syncthreads();  // B blocks, twiddles and D are free for the next column
    }
    if (!ok && t == 0) atomicExch(p.status, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        // a block whose wait gave up has MMAs outstanding: wait for its commit
        // with the full bound before freeing their tensor memory
        if (!ok) mbar_wait(&mbar, (blocks - 1) & 1u);
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"((uint32_t)G::TMEM_ALLOC) : "memory");
    }
}

}  // namespace vspec
