// vspec_tc.cuh — 16-point DFT stages on the 5th-generation tensor cores.
//
// A radix-16 DFT stage (§4's FFT, one pass of it) over a batch of 128 rows is
// one real matrix product
//   [Y_re | Y_im] (128 x 32) = [X_re | X_im] (128 x 32) . F (32 x 32),
//   F[2n][2k] = cos, F[2n][2k+1] = -sin, F[2n+1][2k] = sin, F[2n+1][2k+1] = cos
// of 2 pi n k / 16 (so Y_k = sum_n X_n exp(-2 pi i n k / 16)), interleaving
// re/im along K and N. Each operand is split into bf16 high and low parts,
// x = hi + lo with hi = bf16(x), lo = bf16(x - hi), and three tcgen05.mma
// (kind::f16, bf16 inputs, fp32 accumulation in tensor memory) form
// X_hi F_hi + X_hi F_lo + X_lo F_hi, which carries about 16 significant bits
// of each operand (X_lo F_lo is below that). One thread issues the MMAs;
// tcgen05.commit signals an mbarrier that the CTA waits on with a bounded
// spin; tcgen05.ld brings D back to registers (row m = TMEM lane m).
//
// Shared-memory operand layout (both operands K-major, no swizzle): 8 x 8
// bf16 core matrices of 128 contiguous bytes (8 rows of 16 bytes). Element
// (row r, k) of a 32-wide operand sits at byte
//   (r / 8) * 512 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,
// so the leading-dimension (K) step between core matrices is 128 bytes and the
// stride-dimension (row) step is 512 bytes. A is 128 rows (8 KiB per part),
// B is F^T, 32 rows (2 KiB per part).
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace vspec {
namespace tc {

constexpr int kRows = 128;          // M of one MMA tile
constexpr int kK = 32;              // 16 complex inputs
constexpr int kN = 32;              // 16 complex outputs
constexpr int kAPart = kRows * kK * 2;   // bytes of one bf16 part of A
constexpr int kBPart = kN * kK * 2;      // bytes of one bf16 part of B
constexpr uint32_t kSpinLimit = 1u << 24;  // bounded mbarrier wait

__host__ __device__ constexpr int op_offset(int r, int k) {
    return (r >> 3) * 512 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start >> 4 (bits 0-13), leading byte offset
// >> 4 (16-29), stride byte offset >> 4 (32-45), descriptor version 1
// (46-47), base offset 0, no swizzle (61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;
    return d;
}

// Instruction descriptor of kind::f16: fp32 D (bits 4-5 = 1), bf16 A and B
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t instr_desc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate) : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_addr(mbar)) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_addr(mbar)), "r"(count) : "memory");
}

// Wait for phase `parity` of the mbarrier; gives up after `limit` polls (0:
// gives up at once without polling). Kernels pass the caller's limit to the
// wait for their results and always the full kSpinLimit to the wait that
// drains an outstanding MMA before its tensor memory is freed.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, uint32_t limit = kSpinLimit) {
    const uint32_t a = smem_addr(mbar);
    for (uint32_t it = 0; it < limit; it++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

// Two loads and their wait in one asm statement: 16 lanes x 8 columns,
// repeated 4 times along the columns (tcgen05.ld .16x256b.x4, lanes ta ..
// ta + 15 of the warp's quarter), and 8 columns of this thread's own lane
// (.32x32b.x8 at tw). In the .16x256b fragment thread T holds, for
// repetition i, lane T/4 at columns 8i + 2(T%4) and 8i + 2(T%4) + 1 (v[4i],
// v[4i+1]) and lane T/4 + 8 at the same columns (v[4i+2], v[4i+3]).
__device__ __forceinline__ void tmem_ld_pairs(uint32_t ta, uint32_t tw, float (&v)[16], float (&w)[8]) {
    uint32_t r[24];
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x4.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%24];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%25];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23])
        : "r"(ta), "r"(tw)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
#pragma unroll
    for (int i = 0; i < 8; i++) w[i] = __uint_as_float(r[16 + i]);
}

// Store 16 consecutive columns of this thread's TMEM lane and wait for the
// store to complete (the same thread reads them back later).
__device__ __forceinline__ void tmem_st16_wait(uint32_t taddr, const float (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};\n\t"
        "tcgen05.wait::st.sync.aligned;"
        :: "r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
           "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
           "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
           "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
           "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
           "r"(__float_as_uint(v[15]))
        : "memory");
}

// Split x into bf16 hi + lo.
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// B = F^T in hi and lo parts (row n = output column, K contiguous), from the
// 16-point DFT constants: cos and sin of 2 pi n k / 16 as float2 (re, -im) =
// W_16^(nk) for n, k < 16 in `w16` (w16[(n*k) % 16]).
__device__ __forceinline__ void stage_dft16_operand(unsigned char *bhi, unsigned char *blo,
                                                    const float2 *w16) {
    for (int e = threadIdx.x; e < kN * kK; e += blockDim.x) {
        const int col = e / kK, kk = e % kK;        // D column (output), K index (input)
        const int k = col >> 1, n = kk >> 1;        // complex output k, complex input n
        const float2 w = w16[(n * k) & 15];         // W_16^(nk) = (cos, -sin)
        // F[2n][2k] = c, F[2n][2k+1] = -s, F[2n+1][2k] = s, F[2n+1][2k+1] = c, with w = (c, -s)
        float v;
        if ((kk & 1) == 0) v = (col & 1) ? w.y : w.x;
        else v = (col & 1) ? w.x : -w.y;
        __nv_bfloat16 h, l;
        split_bf16(v, h, l);
        *reinterpret_cast<__nv_bfloat16 *>(bhi + op_offset(col, kk)) = h;
        *reinterpret_cast<__nv_bfloat16 *>(blo + op_offset(col, kk)) = l;
    }
}

// Stage row `r` of A (16 complex inputs v[0..15]) in hi and lo parts.
__device__ __forceinline__ void stage_row(unsigned char *ahi, unsigned char *alo, int r, const float2 (&v)[16]) {
#pragma unroll
    for (int g = 0; g < 4; g++) {  // 8 bf16 (4 complex) per 16-byte chunk of the core-matrix row
        __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            split_bf16(v[4 * g + i].x, h[2 * i], l[2 * i]);
            split_bf16(v[4 * g + i].y, h[2 * i + 1], l[2 * i + 1]);
        }
        *reinterpret_cast<uint4 *>(ahi + op_offset(r, 8 * g)) = *reinterpret_cast<const uint4 *>(h);
        *reinterpret_cast<uint4 *>(alo + op_offset(r, 8 * g)) = *reinterpret_cast<const uint4 *>(l);
    }
}

// Issue the three-term product into TMEM columns [d_col, d_col + 32): K = 32
// takes two K = 16 instructions per term.
__device__ __forceinline__ void issue_dft16(uint32_t d_tmem, const unsigned char *ahi, const unsigned char *alo,
                                            const unsigned char *bhi, const unsigned char *blo, int terms) {
    constexpr uint32_t idesc = instr_desc_bf16(kRows, kN);
    const unsigned char *as[3] = {ahi, ahi, alo};
    const unsigned char *bs[3] = {bhi, blo, bhi};
    uint32_t acc = 0;
    for (int t = 0; t < terms; t++) {
#pragma unroll
        for (int ks = 0; ks < 2; ks++) {  // K = 16 slices: 2 core matrices (256 bytes) apart
            const uint64_t ad = smem_desc(smem_addr(as[t]) + 256u * ks, 128u, 512u);
            const uint64_t bd = smem_desc(smem_addr(bs[t]) + 256u * ks, 128u, 512u);
            mma_bf16(d_tmem, ad, bd, idesc, acc);
            acc = 1;
        }
    }
}

// W_16^m = exp(-2 pi i m / 16) for m < 16, from FP64.
__device__ __forceinline__ void fill_w16(float2 *w16) {
    if (threadIdx.x < 16) {
        double sn, cs;
        sincospi((double)threadIdx.x / 8.0, &sn, &cs);
        w16[threadIdx.x] = make_float2((float)cs, (float)-sn);
    }
}

// Batched 16-point DFTs, y[b][k] = sum_n x[b][n] W_16^(nk), 128 rows per CTA,
// `terms` = 1 (X_hi F_hi) or 3 (hi/lo split). *status is set to 1 if the
// wait for the tensor cores gives up after wait_limit polls; the CTA then
// still waits (with the full bound) for its MMAs to finish before it frees
// their tensor memory.
__global__ void __launch_bounds__(128) dft16_kernel(const float2 *x, float2 *y, int batch, int terms,
                                                    int *status, uint32_t wait_limit) {
    __shared__ __align__(128) unsigned char ops[2 * kAPart + 2 * kBPart];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ float2 w16[16];
    unsigned char *ahi = ops, *alo = ops + kAPart, *bhi = ops + 2 * kAPart, *blo = bhi + kBPart;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long row0 = (long long)blockIdx.x * kRows;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_addr(&tmem_slot)), "r"(32u) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fill_w16(w16);
    __syncthreads();
    stage_dft16_operand(bhi, blo, w16);
    {
        const int r = threadIdx.x;
        float2 v[16];
        const long long b = row0 + r;
#pragma unroll
        for (int n = 0; n < 16; n++) v[n] = b < batch ? x[b * 16 + n] : make_float2(0.f, 0.f);
        stage_row(ahi, alo, r, v);
    }
    fence_proxy_async();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    if (threadIdx.x == 0) {
        issue_dft16(tmem, ahi, alo, bhi, blo, terms);
        mma_commit(&mbar);
    }
    const bool ok = mbar_wait(&mbar, 0, wait_limit);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        float d[32];
        tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16), d);
        const long long b = row0 + 32 * warp + lane;
        if (b < batch) {
#pragma unroll
            for (int k = 0; k < 16; k++) y[b * 16 + k] = make_float2(d[2 * k], d[2 * k + 1]);
        }
    } else if (threadIdx.x == 0) {
        atomicExch(status, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        if (!ok) mbar_wait(&mbar, 0);  // let an outstanding MMA finish before freeing its TMEM
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(32u) : "memory");
    }
}

}  // namespace tc
}  // namespace vspec
