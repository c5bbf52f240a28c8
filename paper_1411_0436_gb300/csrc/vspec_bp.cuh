// vspec_bp.cuh — many banks (beams) in one persistent launch (§3 of arXiv
// 1411.0436: one pipeline per beam; §5: per-launch overheads at small sizes).
//
// One cooperative launch of one 512-thread CTA per SM channelizes every
// bank's call. The work of all banks is one list of tickets in three phases,
// handed out in order by an atomic counter:
//   A: kernel-A tiles of every bank (tile x, spectra [u TA, (u+1) TA)), the
//      register-column forms (PFB: colreg_tile; direct: coldir_tile), into
//      the bank's scratch Z (its whole call);
//   B: row tickets of every bank (row tile x, spectra [u TB, (u+1) TB)): the
//      2048-point row kernel on Z, or for one-row banks (nchan <= 2048) the
//      row transform with the pre-filter on the int8 input; the CTA's two
//      256-thread groups take half the spectra each, sum their detected
//      spectra, and store the sum into set u of the bank's partial sums (one
//      writer per set entry);
//   F: fold tickets of every bank (2048 channels): the sets added in order
//      (compensated) into the caller's accumulator in channel order.
// A bank's B tickets wait (bounded, thread 0) until all its A tickets are
// done, its F tickets until all its B tickets are done. Every wait points to
// tickets of an earlier phase, all CTAs are resident, so the waits end; one
// that gives up raises an abort flag that ends the others and the plan's
// status word reports it. Results do not depend on which CTA ran what.
#pragma once
#include "vspec_ring.cuh"

namespace vspec {

constexpr int kBpMaxBanks = 16;
enum : int { kBpColreg = 0, kBpColdir = 1, kBpRowFir = 2, kBpRow2048Fir = 3 };

struct BpBank {
    ColParams a;             // kernel A's tables and sizes (Z, s0, sc are per ticket)
    RowParams b;             // kernel B's
    void *Z;                 // the call's intermediate: [s][pos][n1] of P2
    float4 *sets;            // partial sums [set][N]
    float4 *acc;             // the caller's accumulator, channel order
    const int *invA, *invB;  // channel k1 N2 + k2 sits at position invA[k2] N1 + invB[k1]
    int form, N2;            // ticket body and column length
    int nspectra;
    int TA, TB;              // spectra per A ticket, per B ticket (even)
    int tilesA, tilesB;      // kernel-A tiles, row tiles
    int nA, nB, nF;          // tickets of each phase
};

struct BpParams {
    BpBank banks[kBpMaxBanks];
    int nbanks;
    int offA[kBpMaxBanks + 1], offB[kBpMaxBanks + 1], offF[kBpMaxBanks + 1];  // first ticket of each bank
    int *ctl;                // [0] ticket counter, [1] abort flag, [2 + 2k] A done, [3 + 2k] B done of bank k
    int *status;             // set to 1 when a wait gives up
    unsigned wait_limit;
};

struct BpTicket {
    int phase;  // 0 A, 1 B, 2 F, -1 past the end
    int bank;
    int i;      // index within the bank's tickets of that phase
};

__device__ __forceinline__ BpTicket bp_decode(const BpParams &q, int t) {
    const int n = q.nbanks;
    const int *off;
    int phase;
    if (t < q.offA[n]) {
        off = q.offA;
        phase = 0;
    } else if (t - q.offA[n] < q.offB[n]) {
        t -= q.offA[n];
        off = q.offB;
        phase = 1;
    } else if (t - q.offA[n] - q.offB[n] < q.offF[n]) {
        t -= q.offA[n] + q.offB[n];
        off = q.offF;
        phase = 2;
    } else {
        return {-1, 0, 0};
    }
    int k = 0;
    while (k + 1 < n && off[k + 1] <= t) k++;
    return {phase, k, t - off[k]};
}

// Thread 0: wait until *ctr >= target (bounded; see ring_wait).
__device__ __forceinline__ bool bp_wait(const BpParams &q, const int *ctr, int target) {
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

// ---------------------------------------------------- one-row banks, FIR --
// Shared memory of one 256-thread group of the one-row body (nchan = N1 <=
// 1024, P taps): the padded row, its N1 accumulators, a ring of P + 1 int8
// frames and the P taps' coefficients.
__host__ __device__ constexpr size_t bp_rowfir_bytes(int N1, int P) {
    return (((size_t)(N1 + (N1 >> 4)) * 16 + (size_t)N1 * 16 + 15) & ~(size_t)15) + (size_t)(P + 1) * N1 * 4 +
           (size_t)P * N1 * 4;
}

// One-row transform with the pre-filter on the int8 input (dual-pol), spectra
// s_beg .. s_end - 1 of the call, by one 256-thread group (the general row
// kernel's passes, row_butterfly): the detected spectra are summed into the
// group's accumulators in shared memory (zeroed here; read by the caller).
template <typename GRP>
__device__ __forceinline__ void bp_rowfir_group(const RowParams &p, int s_beg, int s_end, unsigned char *smem,
                                                GRP grp) {
    using T = P2;
    using A = float4;
    const int tid = grp.tid();
    const int N1 = p.N1, rowstride = N1 + (N1 >> 4);
    T *data = reinterpret_cast<T *>(smem);
    A *acc = reinterpret_cast<A *>(data + rowstride);
    unsigned char *ring = smem + ((((size_t)rowstride * 16 + (size_t)N1 * 16) + 15) & ~(size_t)15);
    float *cfs = reinterpret_cast<float *>(ring + (size_t)(p.P + 1) * N1 * 4);
    auto copy16 = [&](void *dst, const void *src, int bytes) {
        for (int e = tid; e < bytes / 16; e += 256)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                         :: "r"((uint32_t)__cvta_generic_to_shared(static_cast<unsigned char *>(dst) + 16 * e)),
                            "l"(static_cast<const unsigned char *>(src) + 16 * e) : "memory");
    };
    auto stage_frame = [&](long long fr) {  // frame fr into slot fr mod (P + 1)
        copy16(ring + (size_t)(fr % (p.P + 1)) * N1 * 4, p.in + fr * p.N * 4, N1 * 4);
    };
    for (int e = tid; e < N1; e += 256) acc[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (s_beg >= s_end) {
        grp.sync();
        return;
    }
    copy16(cfs, p.coef, p.P * N1 * 4);
    for (int t = 0; t < p.P; t++) stage_frame(s_beg + t);
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int s = s_beg; s < s_end; s++) {
        // the next spectrum's newest frame takes the slot of frame s - 1
        if (s + 1 < s_end) {
            stage_frame(s + p.P);
            asm volatile("cp.async.commit_group;" ::: "memory");
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        grp.sync();  // spectrum s's frames (and the zeroed sums) are visible to the group
        const int slot0 = s % (p.P + 1);
        for (int ip = 0; ip < p.npass; ip++) {
            const Pass ps = p.pass[ip];
            const bool first = ip == 0, last = ip == p.npass - 1;
            const int nb = 1 << (p.lN1 - ps.lr);  // butterflies of the row
            for (int u = tid; u < nb; u += 256) {
                const int b = u >> ps.lm, j = u & (ps.m - 1);
                switch (ps.r) {
                    case 2: row_butterfly<2, 2, false, true>(p, 0, data, acc, nullptr, ps, first, last, 0, b, j, rowstride, nullptr, ring, cfs, slot0); break;
                    case 4: row_butterfly<4, 2, false, true>(p, 0, data, acc, nullptr, ps, first, last, 0, b, j, rowstride, nullptr, ring, cfs, slot0); break;
                    case 8: row_butterfly<8, 2, false, true>(p, 0, data, acc, nullptr, ps, first, last, 0, b, j, rowstride, nullptr, ring, cfs, slot0); break;
                    default: row_butterfly<16, 2, false, true>(p, 0, data, acc, nullptr, ps, first, last, 0, b, j, rowstride, nullptr, ring, cfs, slot0); break;
                }
            }
            grp.sync();
        }
    }
}

// ------------------------------------------------------------- tickets --
// Kernel-A ticket i of a bank: tile x = i mod tilesA (adjacent tiles, which
// share the input's lines, run together) over spectra range u = i / tilesA.
__device__ __forceinline__ void bp_ticket_a(const BpBank &bk, int i, unsigned char *smem) {
    const int x = i % bk.tilesA, u = i / bk.tilesA;
    const int s_beg = u * bk.TA, s_end = min(bk.nspectra, s_beg + bk.TA);
    const ColParams &p = bk.a;
    if (bk.form == kBpColreg) {
        switch (bk.N2) {
            case 2: colreg_tile<2, 2>(p, bk.Z, 0, bk.nspectra, x, s_beg, s_end, smem, true); break;
            case 4: colreg_tile<4, 4>(p, bk.Z, 0, bk.nspectra, x, s_beg, s_end, smem, true); break;
            case 8: colreg_tile<8, 8>(p, bk.Z, 0, bk.nspectra, x, s_beg, s_end, smem, true); break;
            case 16: colreg_tile<16, 16>(p, bk.Z, 0, bk.nspectra, x, s_beg, s_end, smem, true); break;
            case 32: colreg_tile<32, 8>(p, bk.Z, 0, bk.nspectra, x, s_beg, s_end, smem, true); break;
            case 64: colreg_tile<64, 8>(p, bk.Z, 0, bk.nspectra, x, s_beg, s_end, smem, true); break;
            default: colreg_tile<128, 8>(p, bk.Z, 0, bk.nspectra, x, s_beg, s_end, smem, true); break;
        }
    } else {
        switch (bk.N2) {
            case 2: coldir_tile<2>(p, bk.Z, 0, bk.nspectra, x, s_beg, s_end, smem, true); break;
            case 4: coldir_tile<4>(p, bk.Z, 0, bk.nspectra, x, s_beg, s_end, smem, true); break;
            case 8: coldir_tile<8>(p, bk.Z, 0, bk.nspectra, x, s_beg, s_end, smem, true); break;
            case 16: coldir_tile<16>(p, bk.Z, 0, bk.nspectra, x, s_beg, s_end, smem, true); break;
            case 32: coldir_tile<32>(p, bk.Z, 0, bk.nspectra, x, s_beg, s_end, smem, true); break;
            case 64: coldir_tile<64>(p, bk.Z, 0, bk.nspectra, x, s_beg, s_end, smem, true); break;
            case 128: coldir_tile<128>(p, bk.Z, 0, bk.nspectra, x, s_beg, s_end, smem, true); break;
            default: coldir_tile<256>(p, bk.Z, 0, bk.nspectra, x, s_beg, s_end, smem, true); break;
        }
    }
}

// The two groups' spectra of a kernel-B ticket: group 0 the first h (even),
// group 1 the rest of [s0, s1).
__device__ __forceinline__ void bp_halves(int s0, int s1, int g, int *b0, int *b1) {
    const int T = s1 - s0;
    const int h = min(T, (T + 1) / 2 + (((T + 1) / 2) & 1));
    *b0 = g ? s0 + h : s0;
    *b1 = g ? s1 : s0 + h;
}

// Kernel-B ticket i of a bank: row tile x = i mod tilesB over spectra range
// u = i / tilesB, stored into set u.
template <bool FIR>
__device__ __forceinline__ void bp_ticket_b2048(const BpBank &bk, int i, unsigned char *smem) {
    using A = float4;
    const int x = i % bk.tilesB, u = i / bk.tilesB;
    const int g = threadIdx.x >> 8, tid = threadIdx.x & 255;
    int s_beg, s_end;
    bp_halves(u * bk.TB, min(bk.nspectra, (u + 1) * bk.TB), g, &s_beg, &s_end);
    const RowGrp2 grp{g};
    P2 *rows = reinterpret_cast<P2 *>(smem + g * 2 * (size_t)kRow2048Stride * sizeof(P2));
    const int half = tid >> 7, ht = tid & 127;
    A acc[8], comp[8];
#pragma unroll
    for (int e = 0; e < 8; e++) acc[e] = comp[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int s = s_beg; s < s_end; s += 2) {
        const bool two = s + 1 < s_end;
        if (half == 0 || two)
            row2048_first<2, false, FIR, false, true>(bk.b, bk.Z, bk.nspectra, rows + half * kRow2048Stride, x,
                                                       s + half, ht, half, grp);
        grp.sync();
        row2048_last<2, false>(rows, tid, acc, comp);
        if (two) row2048_last<2, false>(rows + kRow2048Stride, tid, acc, comp);
        grp.sync();
    }
    __syncthreads();  // both groups are done with their rows
    A *xch = reinterpret_cast<A *>(smem);  // group 1's sums, [e][tid]
    if (g == 1) {
#pragma unroll
        for (int e = 0; e < 8; e++) xch[e * 256 + tid] = acc[e];
    }
    __syncthreads();
    if (g == 0) {
        A *pt = bk.sets + (size_t)u * bk.b.N + (size_t)x * 2048 + 8 * tid;
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const A w = xch[e * 256 + tid];
            pt[e] = make_float4(acc[e].x + w.x, acc[e].y + w.y, acc[e].z + w.z, acc[e].w + w.w);
        }
    }
}

// Kernel-B ticket u of a one-row bank (nchan <= 1024): spectra range u.
__device__ __forceinline__ void bp_ticket_rowfir(const BpBank &bk, int u, unsigned char *smem) {
    using A = float4;
    const RowParams &p = bk.b;
    const int g = threadIdx.x >> 8;
    const size_t gbytes = (bp_rowfir_bytes(p.N1, p.P) + 15) & ~(size_t)15;
    int s_beg, s_end;
    bp_halves(u * bk.TB, min(bk.nspectra, (u + 1) * bk.TB), g, &s_beg, &s_end);
    bp_rowfir_group(p, s_beg, s_end, smem + g * gbytes, RowGrp2{g});
    __syncthreads();
    // accumulator e = q U + b holds position b RL + q (U = N1 / RL)
    const A *a0 = reinterpret_cast<const A *>(smem + (size_t)(p.N1 + (p.N1 >> 4)) * 16);
    const A *a1 = reinterpret_cast<const A *>(smem + gbytes + (size_t)(p.N1 + (p.N1 >> 4)) * 16);
    const int lq = p.lN1 - p.pass[p.npass - 1].lr, RL = p.pass[p.npass - 1].r;
    A *pt = bk.sets + (size_t)u * p.N;
    for (int e = threadIdx.x; e < p.N1; e += 512) {
        const int q = e >> lq, b = e & ((1 << lq) - 1);
        const A v = a0[e], w = a1[e];
        pt[b * RL + q] = make_float4(v.x + w.x, v.y + w.y, v.z + w.z, v.w + w.w);
    }
}

// Fold ticket i of a bank: channels kBpFoldChannels i .. + kBpFoldChannels -
// 1, every set in order (compensated), added into the caller's accumulator.
constexpr int kBpFoldChannels = 2048;
__device__ __forceinline__ void bp_ticket_fold(const BpBank &bk, int i) {
    const int N = bk.b.N, N1 = bk.b.N1, N2 = bk.N2;
    const int nsets = (bk.nspectra + bk.TB - 1) / bk.TB;
    for (int k = i * kBpFoldChannels + threadIdx.x; k < min(N, (i + 1) * kBpFoldChannels); k += 512) {
        const int k1 = k / N2, k2 = k - k1 * N2;
        const size_t pos = (size_t)__ldg(bk.invA + k2) * N1 + __ldg(bk.invB + k1);
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f), c = s;
        for (int u = 0; u < nsets; u++) kahan_add(s, c, __ldcg(bk.sets + (size_t)u * N + pos));
        kahan_settle(s, c);
        const float4 o = bk.acc[k];
        bk.acc[k] = make_float4(o.x + s.x, o.y + s.y, o.z + s.z, o.w + s.w);
    }
}

#ifdef VSPEC_DEFINE_BP_KERNEL  // defined in one translation unit (vspec_bp.cu)
__global__ void __launch_bounds__(512, 1) bp_kernel(const __grid_constant__ BpParams q) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_t, s_ok;
    const int total = q.offA[q.nbanks] + q.offB[q.nbanks] + q.offF[q.nbanks];
    // Thread 0 holds the next ticket, fetched while the current one runs,
    // and whether its producers were already done when it looked (counters
    // only grow, so a yes stays true). A CTA's prefetched ticket is later
    // than its current one, so the earliest unfinished ticket is always some
    // CTA's current ticket and can run.
    int next = 0;
    bool next_ready = false;
    auto producers = [&](const BpTicket &k, const int **ctr, int *target) {
        const BpBank &bk = q.banks[k.bank];
        *ctr = k.phase == 1 ? q.ctl + 2 + 2 * k.bank : q.ctl + 3 + 2 * k.bank;
        *target = k.phase == 1 ? bk.nA : bk.nB;
        return k.phase == 1 || k.phase == 2;
    };
    if (threadIdx.x == 0) next = atomicAdd(q.ctl, 1);
    for (;;) {
        bool cur_ready = false;  // thread 0 only (shared s_ok is written only between the two barriers)
        if (threadIdx.x == 0) {
            s_t = next;
            cur_ready = next_ready;
            next = atomicAdd(q.ctl, 1);
        }
        __syncthreads();
        const int t = s_t;
        if (t >= total) break;
        const BpTicket k = bp_decode(q, t);
        const BpBank &bk = q.banks[k.bank];
        int *doneA = q.ctl + 2 + 2 * k.bank, *doneB = doneA + 1;
        if (threadIdx.x == 0) {
            bool ok = k.phase >= 0;
            const int *ctr;
            int target;
            if (ok && !cur_ready && producers(k, &ctr, &target)) ok = bp_wait(q, ctr, target);
            s_ok = ok;
            // look at the next ticket's producers now; the answer is used next time
            next_ready = false;
            if (next < total) {
                const BpTicket kn = bp_decode(q, next);
                next_ready = !producers(kn, &ctr, &target) || ld_acquire_gpu(ctr) >= target;
            }
        }
        __syncthreads();
        if (!s_ok) continue;  // aborted: skip what is left
        if (k.phase == 0) bp_ticket_a(bk, k.i, smem_raw);
        else if (k.phase == 1) {
            if (bk.form == kBpRowFir) bp_ticket_rowfir(bk, k.i, smem_raw);
            else if (bk.form == kBpRow2048Fir) bp_ticket_b2048<true>(bk, k.i, smem_raw);
            else bp_ticket_b2048<false>(bk, k.i, smem_raw);
        } else {
            bp_ticket_fold(bk, k.i);
        }
        __syncthreads();  // the ticket's stores are issued; shared memory is free
        if (threadIdx.x == 32 && k.phase < 2) {  // warp 1 signals while warp 0 takes the next ticket
            __threadfence();
            atomicAdd(k.phase == 0 ? doneA : doneB, 1);
        }
    }
}
#endif  // VSPEC_DEFINE_BP_KERNEL

}  // namespace vspec
