// vspec_ring.cuh — the persistent form of the two-kernel path (§4 loop:
// pre-filter, FFT, detect, accumulate) with its four-step intermediate in a
// ring of chunk slots small enough to stay in L2.
//
// One cooperative launch of one 512-thread CTA per SM. The call's spectra are
// cut into slots of S spectra; slot c's intermediate lives in ring slot
// c mod R. The work is a list of tickets in a fixed order, handed out by an
// atomic counter:
//   A(0) .. A(L-1), then for c = 0, 1, ...: B(c), A(c + L)
// where A(c) is the kernel-A tiles of slot c (pre-filter, column DFTs,
// twiddles, into the ring slot) and B(c) the kernel-B tickets of slot c (row
// DFTs, detection, sums). A CTA runs one ticket at a time; before it starts,
// thread 0 waits (bounded) until
//   A(c): every B ticket of slot c - R is done (the ring slot is free);
//   B(c): every A ticket of slot c is done, and every B ticket of slot c - K
//         (the previous writer of the same partial-sum sets).
// Every dependency points to tickets handed out earlier, and all CTAs are
// resident (cooperative launch), so the earliest unfinished ticket can always
// run: the waits end. A wait that passes its poll limit sets an abort flag
// (and the plan's status word); every other wait then returns at once and
// the remaining tickets are skipped, so the launch ends.
//
// A B ticket covers T = S / V spectra of one 2048-point row tile; its two
// 256-thread groups take the two halves, sum their detected spectra in
// registers, and group 1 hands its sums to group 0 through shared memory, so
// each ticket makes one flush into set (c mod K) V + v of the partial sums
// (stored by the set's first writer, slots c < K, else added in L2). The
// order of additions into a set is the slot order, so results do not depend
// on which CTA ran what: the fold after the launch adds the sets in order.
#pragma once
#include "vspec_kernels.cuh"

namespace vspec {

struct RingParams {
    ColParams a;          // kernel A's tables and sizes (its Z, s0 and sc are per ticket)
    RowParams b;          // kernel B's tables and sizes (its Z, partial and sc are per ticket)
    void *ring;           // R slots of S spectra: [slot][s][pos][n1] of P2
    void *sets;           // partial sums [set][N] of float4, set = (c mod K) V + v
    int *ctl;             // [0] ticket counter, [1] abort flag, [2, 2 + nslot) A done, then B done
    int *status;          // set to 1 when a wait gives up
    unsigned wait_limit;  // polls of one wait (about 100 ns each)
    int nspectra;         // spectra of this launch
    long long s0;         // this launch's first spectrum within the call's input
    int S, R, L, V, K;    // spectra per slot, ring slots, lookahead (slots), B tickets per row, set cycle
    int nslot;            // slots of this launch
    int c0;               // global index of this launch's first slot
    int tilesA, tilesB;   // kernel-A tiles, 2048-point row tiles
    int discard;          // drop each consumed row of the ring from L2 without writing it back
};

struct RingTicket {
    int kind;  // 0: A, 1: B, -1: past the end
    int c;     // slot
    int i;     // A: tile; B: row tile * V + part
};

__device__ __forceinline__ RingTicket ring_decode(const RingParams &q, int nA, int nB, long long t) {
    const int Lp = min(q.L, q.nslot);
    const long long pre = (long long)Lp * nA;
    if (t < pre) return {0, (int)(t / nA), (int)(t % nA)};
    t -= pre;
    const int mid = q.nslot - Lp;
    const long long blk = (long long)nA + nB;
    if (t < (long long)mid * blk) {
        const int c = (int)(t / blk), r = (int)(t % blk);
        if (r < nB) return {1, c, r};
        return {0, c + Lp, r - nB};
    }
    t -= (long long)mid * blk;
    if (t < (long long)Lp * nB) return {1, mid + (int)(t / nB), (int)(t % nB)};
    return {-1, 0, 0};
}

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0: wait until *ctr >= target. False if the launch was aborted or
// this wait gave up (which aborts it).
__device__ __forceinline__ bool ring_wait(const RingParams &q, const int *ctr, int target) {
    int *abort_flag = q.ctl + 1;
    for (unsigned n = 0;; n++) {
        if (ld_acquire_gpu(ctr) >= target) return true;
        if (*(volatile int *)abort_flag) return false;
        if (n >= q.wait_limit) {
            atomicExch(abort_flag, 1);
            if (q.status) atomicExch(q.status, 1);
            return false;
        }
        __nanosleep(100);
    }
}

// Drop the 128-byte lines [p, p + bytes) from L2 without writing them back
// (their contents become undefined; the next writer of the ring slot
// overwrites them).
__device__ __forceinline__ void discard_l2(const void *p) {
    asm volatile("discard.global.L2 [%0], 128;" :: "l"(p) : "memory");
}

template <int N2, int R1>
struct RingShape {
    static constexpr size_t rows_bytes = 2 * (size_t)kRow2048Stride * sizeof(P2);  // one B group's two rows
    static constexpr size_t smem = ColReg<N2, R1>::smem > 2 * rows_bytes ? ColReg<N2, R1>::smem : 2 * rows_bytes;
};

template <int N2, int R1>
__global__ void __launch_bounds__(512, 1) ring_kernel(const __grid_constant__ RingParams q) {
    using A = float4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long s_t;
    __shared__ int s_ok;
    const int nA = q.tilesA, nB = q.tilesB * q.V;
    const long long total = (long long)q.nslot * (nA + nB);
    int *doneA = q.ctl + 2, *doneB = q.ctl + 2 + q.nslot;
    const size_t slot_elems = (size_t)q.S * q.b.N;
    bool twc_loaded = false;
    // (tickets are fetched when the CTA is free: a ticket fetched ahead would
    // wait behind the current one and hold back the slot it frees)
    for (;;) {
        if (threadIdx.x == 0) s_t = atomicAdd(q.ctl, 1);
        __syncthreads();
        const long long t = s_t;
        if (t >= total) break;
        const RingTicket k = ring_decode(q, nA, nB, t);
        if (threadIdx.x == 0) {
            bool ok = k.kind >= 0;
            if (k.kind == 0) {
                if (k.c >= q.R) ok = ring_wait(q, doneB + (k.c - q.R), nB);
            } else if (k.kind == 1) {
                ok = ring_wait(q, doneA + k.c, nA);
                if (ok && k.c >= q.K) ok = ring_wait(q, doneB + (k.c - q.K), nB);
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) continue;  // aborted: skip what is left
        const int sc = min(q.S, q.nspectra - k.c * q.S);
        P2 *zc = reinterpret_cast<P2 *>(q.ring) + (size_t)(k.c % q.R) * slot_elems;
        if (k.kind == 0) {
            // the first-pass twiddles stay loaded until a B ticket overwrites shared memory
            colreg_tile<N2, R1>(q.a, zc, q.s0 + (long long)k.c * q.S, sc, k.i, 0, sc, smem_raw, !twc_loaded);
            twc_loaded = true;
        } else {
            twc_loaded = false;
            const int x = k.i / q.V, v = k.i % q.V;
            const int T = q.S / q.V;
            const int g = threadIdx.x >> 8, tid = threadIdx.x & 255;
            const int h = (T + 1) / 2 + ((T + 1) / 2 & 1);  // group 0's share, even (whole pairs)
            const int b0 = v * T + (g ? min(h, T) : 0), b1 = v * T + (g ? T : min(h, T));
            const int s_beg = min(b0, sc), s_end = min(b1, sc);
            const RowGrp2 grp{g};
            P2 *rows = reinterpret_cast<P2 *>(smem_raw + g * RingShape<N2, R1>::rows_bytes);
            const int half = tid >> 7, ht = tid & 127;
            A acc[8], comp[8];
#pragma unroll
            for (int e = 0; e < 8; e++) acc[e] = comp[e] = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int s = s_beg; s < s_end; s += 2) {
                const bool two = s + 1 < s_end;
                if (half == 0 || two) {
                    row2048_first<2, false, false, false, true>(q.b, zc, sc, rows + half * kRow2048Stride, x,
                                                                  s + half, ht, half, grp);
                    if (q.discard) {  // every load of this row is done (the half barrier)
                        const char *zr = reinterpret_cast<const char *>(zc + (size_t)(s + half) * q.b.N +
                                                                        (size_t)x * 2048);
                        discard_l2(zr + (size_t)ht * 256);
                        discard_l2(zr + (size_t)ht * 256 + 128);
                    }
                }
                grp.sync();
                row2048_last<2, false>(rows, tid, acc, comp);
                if (two) row2048_last<2, false>(rows + kRow2048Stride, tid, acc, comp);
                grp.sync();
            }
            __syncthreads();  // both groups are done with their rows
            A *xch = reinterpret_cast<A *>(smem_raw);  // group 1's sums, [e][tid]
            if (g == 1) {
#pragma unroll
                for (int e = 0; e < 8; e++) xch[e * 256 + tid] = acc[e];
            }
            __syncthreads();
            if (g == 0) {
                const int cg = q.c0 + k.c;
                const int set = (cg % q.K) * q.V + v;
                A *pt = reinterpret_cast<A *>(q.sets) + (size_t)set * q.b.N + (size_t)x * 2048 + 8 * tid;
#pragma unroll
                for (int e = 0; e < 8; e++) {
                    const A w = xch[e * 256 + tid];
                    const A sum = make_float4(acc[e].x + w.x, acc[e].y + w.y, acc[e].z + w.z, acc[e].w + w.w);
                    if (cg < q.K) pt[e] = sum;  // the set's first writer
                    else atomicAdd(pt + e, sum);
                }
            }
        }
        __syncthreads();  // the ticket's stores are issued; shared memory is free
        if (threadIdx.x == 32) {  // warp 1 signals while warp 0 takes the next ticket
            __threadfence();
            atomicAdd((k.kind == 0 ? doneA : doneB) + k.c, 1);
        }
    }
}

}  // namespace vspec
