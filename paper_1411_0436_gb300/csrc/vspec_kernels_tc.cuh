// vspec_kernels_tc.cuh — row-DFT kernel whose first radix-16 pass runs on the
// tensor cores.
//
// Same work as rowfft_detect_kernel (row DFTs of length N1 = 2048 over a
// group of spectra, detection and accumulation, §4), but the first
// decimation-in-frequency pass, 128 radix-16 butterflies per row and
// polarisation, is one 128 x 32 x 32 tensor-core product per polarisation
// (vspec_tc.cuh: bf16 hi/lo operands, three MMAs, fp32 accumulation in
// tensor memory). Its outputs are multiplied by the pass twiddles on the CUDA
// cores and the remaining passes run as in the FP32 kernel.
#pragma once
#include "vspec_kernels.cuh"
#include "vspec_tc.cuh"

namespace vspec {

struct TcStatus {
    int *status;          // set to 1 if a bounded wait for the tensor cores gave up
    uint32_t wait_limit;  // polls of that wait (the drain before freeing TMEM always has the full bound)
};

constexpr int kTcN1 = 2048;
constexpr int kTcSmemOps = 4 * tc::kAPart + 2 * tc::kBPart;  // A0/A1 hi, lo and F hi, lo

__host__ __device__ constexpr size_t tc_rowfft_smem(bool kahan) {
    return (size_t)kTcSmemOps + (size_t)(kTcN1 + kTcN1 / 16) * 16 + (size_t)kTcN1 * 16 * (kahan ? 2 : 1);
}

template <int TERMS, bool KAHAN = false>
__global__ void __launch_bounds__(256, 1) rowfft_detect_tc_kernel(const __grid_constant__ RowParams p,
                                                                  TcStatus ts) {
    using namespace tc;
    extern __shared__ __align__(128) unsigned char smem_tc[];
    unsigned char *a0hi = smem_tc, *a0lo = a0hi + kAPart, *a1hi = a0lo + kAPart, *a1lo = a1hi + kAPart;
    unsigned char *bhi = a1lo + kAPart, *blo = bhi + kBPart;
    P2 *data = reinterpret_cast<P2 *>(smem_tc + kTcSmemOps);   // one row, padded
    const int rowstride = kTcN1 + kTcN1 / 16;
    float4 *acc = reinterpret_cast<float4 *>(data + rowstride);
    float4 *comp = acc + kTcN1;  // compensation (compensated plans only)
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ float2 w16[16];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_addr(&tmem_slot)), "r"(64u) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fill_w16(w16);
    __syncthreads();
    stage_dft16_operand(bhi, blo, w16);
    fence_proxy_async();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const Pass p0 = p.pass[0];  // radix 16, block length 2048, 128 butterflies
    bool ok = true;
    uint32_t parity = 0;
    int k = 0;  // MMA batches issued so far (mbarrier phase)
    const int RL = p.pass[p.npass - 1].r;
    const int U = kTcN1 >> p.pass[p.npass - 1].lr;

    const Span sp = block_span(p.tiles, p.sc);
    for (long long f = sp.lo; f < sp.hi && ok;) {
        const int x = (int)(f / p.sc);  // row
        const long long base = (long long)x * p.sc;
        const int s_beg = (int)(f - base);
        const int s_end = (int)(min(sp.hi, base + p.sc) - base);
        f = base + s_end;
        for (int e = tid; e < kTcN1; e += blockDim.x) {
            acc[e] = make_float4(0.f, 0.f, 0.f, 0.f);
            if constexpr (KAHAN) comp[e] = acc[e];
        }
        __syncthreads();

        for (int s = s_beg; s < s_end && ok; s++, k++) {
            const P2 *zr = reinterpret_cast<const P2 *>(p.Z) + (size_t)s * p.N + (size_t)x * kTcN1;
            if (tid < kRows) {
                float2 v0[16], v1[16];  // X and Y as (re, im)
#pragma unroll
                for (int r = 0; r < 16; r++) {
                    const P2 e = zr[tid + kRows * r];
                    v0[r] = make_float2(e.re.x, e.im.x);
                    v1[r] = make_float2(e.re.y, e.im.y);
                }
                stage_row(a0hi, a0lo, tid, v0);
                stage_row(a1hi, a1lo, tid, v1);
            }
            fence_proxy_async();
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (tid == 0) {
                issue_dft16(tmem, a0hi, a0lo, bhi, blo, TERMS);
                issue_dft16(tmem + 32u, a1hi, a1lo, bhi, blo, TERMS);
                mma_commit(&mbar);
            }
            parity = (uint32_t)(k & 1);
            ok = mbar_wait(&mbar, parity, ts.wait_limit);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (ok && warp < 4) {
                float d0[32], d1[32];
                tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16), d0);
                tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + 32u, d1);
                const int j = 32 * warp + lane;
                const float2 *tw = p.twB + p0.off + j * 15;
#pragma unroll
                for (int q = 0; q < 16; q++) {
                    P2 vq = make_p2(d0[2 * q], d0[2 * q + 1], d1[2 * q], d1[2 * q + 1]);
                    if (q > 0) vq = cmul(vq, __ldg(tw + q - 1));
                    data[pad16(j + kRows * q)] = vq;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            ok = __syncthreads_and(ok);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!ok) break;
            for (int ip = 1; ip < p.npass; ip++) {
                const Pass ps = p.pass[ip];
                const bool last = ip == p.npass - 1;
                const int per_row = kTcN1 >> ps.lr;
                for (int u = tid; u < per_row; u += blockDim.x) {
                    const int b = u >> ps.lm, jj = u & (ps.m - 1);
                    switch (ps.r) {
                        case 2: row_butterfly<2, 2, KAHAN>(p, x, data, acc, nullptr, ps, false, last, 0, b, jj, rowstride, comp); break;
                        case 4: row_butterfly<4, 2, KAHAN>(p, x, data, acc, nullptr, ps, false, last, 0, b, jj, rowstride, comp); break;
                        case 8: row_butterfly<8, 2, KAHAN>(p, x, data, acc, nullptr, ps, false, last, 0, b, jj, rowstride, comp); break;
                        default: row_butterfly<16, 2, KAHAN>(p, x, data, acc, nullptr, ps, false, last, 0, b, jj, rowstride, comp); break;
                    }
                }
                __syncthreads();
            }
        }
        if (!ok) break;

        // flush into this block's slot: accumulator slot e = q * U + b holds position b * RL + q
        const size_t so = (size_t)span_slot(p.tiles, p.sc, x) * p.N + (size_t)x * kTcN1;
        float4 *part = reinterpret_cast<float4 *>(p.partial) + so;
        for (int e = tid; e < kTcN1; e += blockDim.x) {
            const int q = e >> (11 - p.pass[p.npass - 1].lr), b = e & (U - 1);
            float4 a = part[b * RL + q];
            if constexpr (KAHAN) {
                float4 *pc = reinterpret_cast<float4 *>(p.partial_comp) + so;
                float4 c = pc[b * RL + q];
                kahan_add(a, c, sub4(acc[e], comp[e]));
                pc[b * RL + q] = c;
                part[b * RL + q] = a;
            } else {
                const float4 d = acc[e];
                part[b * RL + q] = make_float4(a.x + d.x, a.y + d.y, a.z + d.z, a.w + d.w);
            }
        }
        __syncthreads();  // acc is zeroed again by the next segment
    }
    if (!ok && tid == 0) atomicExch(ts.status, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        // the MMAs of the batch whose wait gave up are still outstanding: wait
        // for that commit with the full bound before freeing their TMEM (one
        // batch is under a microsecond of tensor-core work, so only a stopped
        // tensor pipe could outlast the bound)
        if (!ok) mbar_wait(&mbar, parity);
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(64u) : "memory");
    }
}

}  // namespace vspec
