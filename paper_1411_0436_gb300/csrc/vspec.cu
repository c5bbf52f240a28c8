// vspec.cu — host side of the C ABI declared in include/vspec.h.
//
// Plan creation follows the initialisation steps of §4 of arXiv 1411.0436
// (load the filter coefficients, create the FFT plan); execution follows its
// processing loop (pre-filter, FFTs, accumulate) and the dump its final copy
// to the host. The device code is in vspec_kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "vspec.h"
#include "vspec_fused.cuh"
#include "vspec_fused_w.cuh"
#include "vspec_kernels.cuh"
#include "vspec_tc.cuh"
#include "vspec_kernels_tc.cuh"
#include "vspec_kernels_coltc.cuh"
#include "vspec_kernels_tcfir.cuh"
#include "vspec_ring.cuh"
#include "vspec_bp.cuh"
#include "vspec_internal.h"

using vspec::Pass;

// vspec_ring.cu
const void *vspec_pick_kernel_ring(int N2, size_t *smem);
cudaError_t vspec_ring_debug_flags(unsigned *flags, bool clear);
// vspec_bp.cu
const void *vspec_bp_kernel();
size_t vspec_bp_smem_a(int form, int N2);
size_t vspec_bp_smem_b(int form, int N1, int P);
cudaError_t vspec_bp_debug_flags(unsigned *flags, bool clear);

namespace {

thread_local std::string g_last_error;

// Polls of the bounded device-side waits for results (vspec_set_wait_limit).
std::atomic<uint32_t> g_wait_limit{vspec::tc::kSpinLimit};

vspec_status cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return VSPEC_ERR_CUDA;
}

#define VSPEC_CUDA(call)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

// The dynamic shared-memory cap is a property of the kernel function, shared
// by every plan that launches it: only ever raise it, never lower it.
std::mutex g_smem_attr_mu;
cudaError_t raise_smem_cap(const void *fn, size_t bytes) {
    std::lock_guard<std::mutex> lock(g_smem_attr_mu);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
int ilog2(long long v) {
    int e = 0;
    while ((1LL << e) < v) e++;
    return e;
}

// Radices of a length-2^e DFT: passes of at most maxbits bits, as even as
// possible.
std::vector<int> radix_list(int e, int maxbits = 4) {
    std::vector<int> r;
    if (e == 0) return r;
    const int np = (e + maxbits - 1) / maxbits;
    for (int i = 0; i < np; i++) {
        const int bits = e / np + (i < e % np ? 1 : 0);
        r.push_back(1 << bits);
    }
    return r;
}

// DIF pass descriptors and twiddle-table offsets for a length-L transform.
std::vector<Pass> make_passes(int L, const std::vector<int> &radices, int *tw_entries) {
    std::vector<Pass> ps;
    int lb = L, off = 0;
    for (int r : radices) {
        Pass p;
        p.r = r;
        p.lb = lb;
        p.m = lb / r;
        p.off = off;
        p.lr = ilog2(r);
        p.lm = ilog2(p.m);
        off += p.m * (r - 1);
        ps.push_back(p);
        lb /= r;
    }
    *tw_entries = off;
    return ps;
}

// Output index held by in-place position pos after the DIF passes:
// pos = sum_i q_i * M_i  ->  k = q_1 + r_1 (q_2 + r_2 (...)).
std::vector<int> digit_reverse(int L, const std::vector<int> &radices) {
    std::vector<int> k_of_pos(L);
    for (int pos = 0; pos < L; pos++) {
        int rem = pos, lb = L, k = 0, scale = 1;
        for (int r : radices) {
            const int m = lb / r;
            const int q = rem / m;
            rem -= q * m;
            k += q * scale;
            scale *= r;
            lb = m;
        }
        k_of_pos[pos] = k;
    }
    return k_of_pos;
}

}  // namespace

struct vspec_plan {
    int N = 0, P = 0, npol = 0, mode = 0, window = 0, device = 0;
    int N1 = 0, N2 = 0, C = 0, PT = 0, PPT = 0, TA = 0, RB = 0, TB = 0;
    int tileG = 1;                   // kernel-A tiles per group (tile_split)
    int req_n2 = 0, req_cols = 0;    // requested column length / kernel-A tile columns (0: the plan's choice)
    const char *formA = "general";   // kernel A's form (vspec_plan_describe)
    const char *formB = "general";   // kernel B's form
    int num_sms = 0, occA = 1, occB = 1;
    int sc_max = 1;                  // spectra per chunk
    int sc_cap = 1, slots_cap = 1;   // largest chunk a tuning may ask for; slots allocated
    int sc_alloc = 1;                // chunk spectra the scratch holds now
    int blocks_a = 0, blocks_b = 0;  // CTAs per kernel-A / kernel-B launch, 0: one wave
    bool fir_b = false;              // one-row transform: kernel B only, FIR in its first pass
    bool fold2048 = false;           // the fold runs reduce2048_kernel (2048-point rows, N2 >= 16)
    bool gather = false;             // long PFB: kernel A reads the FIR taps from the input
    size_t smemA = 0, smemB = 0;
    std::vector<Pass> passA, passB;
    float *coef = nullptr;
    float2 *twA = nullptr, *twB = nullptr, *twZ = nullptr;
    int *invA = nullptr, *invB = nullptr;
    void *Z = nullptr, *partial = nullptr;
    size_t scratch_bytes = 0;
    const void *kernelA = nullptr, *kernelB = nullptr, *kernelR = nullptr;
    // fused one-pass path (dual-pol, 2048..32768 channels)
    bool fused = false, fused_w = false;
    int logn1 = 0, cluster = 1, nclusters = 1;
    size_t smemF = 0;
    const void *kernelF = nullptr;
    unsigned flags = 0;
    // fused plans: a two-kernel plan that channelizes a share of the spectra
    // on the SMs the clusters leave idle, concurrently with the fused kernel
    vspec_plan *assist = nullptr;
    vspec_plan *owner = nullptr;  // the plan whose profiling records this plan's launches
    int assist_permille = 0;
    int two_kernel_from = INT_MAX;  // fused plans: calls with this many spectra use `assist` alone
    int prio_high = 0;            // greatest stream priority of the device
    cudaStream_t assist_st = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_main = nullptr, ev_assist = nullptr;
    bool tc = false;           // first row pass on the tensor cores
    bool tc_cols = false;      // column DFTs (kernel A) on the tensor cores
    bool tc_int8 = false;      // ... with the pre-filter, on the int8 input (per-column operands)
    int bterms = 1;            // their coefficient parts (fp16 hi, or hi and lo)
    unsigned char *dftop = nullptr;  // their DFT operand (fp16 hi, lo)
    bool kahan = false;        // compensated accumulation at every level
    void *partial_comp = nullptr, *out_comp = nullptr;
    int *tc_status = nullptr;  // bounded-wait flag of the tensor-core or ring kernel
    // persistent ring form (VSPEC_PLAN_RING): Z holds ringR slots of ringS
    // spectra, `partial` ring_sets partial-sum sets
    bool ring = false;
    int ringS = 0, ringR = 0, ringL = 0, ringV = 0;  // spectra per slot, slots, lookahead, B tickets per row
    int ring_sets = 0;
    int ring_discard = 1;        // drop consumed ring rows from L2 without a write-back
    int ring_stall = -1;         // failure injection: the next launch's B tickets of this slot never start
    int *ring_ctl = nullptr;     // ticket counter, abort flag, per-slot done counters
    const void *kernelRing = nullptr;
    size_t smemRing = 0;
    int ring_grid = 0;           // CTAs of a ring launch (all resident)
    // sub-bands: input [time][nsub][pol][re, im], output [nsub][nchan]
    int nsub = 1;
    int sb_chunk = 0;          // spectra per de-interleaved chunk
    int8_t *sb_scratch = nullptr;
    // instrumentation (vspec_plan_set_profiling)
    struct Rec {
        int kind;
        int spectra;
        cudaEvent_t start, stop;
    };
    bool profiling = false;
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> event_pool;
    // host-input pipeline (vspec_execute_host), created on first use
    bool host_ready = false;
    int host_mode = VSPEC_HOST_STAGED;
    size_t host_chunk_bytes = 0;  // staged chunk of input bytes; 0: sized from the first call
    size_t host_bytes = 0;  // device memory of the host pipeline
    cudaStream_t copy_st = nullptr, comp_st = nullptr;
    cudaEvent_t ev_start = nullptr, ev_done = nullptr;
    cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_used[2] = {nullptr, nullptr};
    int8_t *stage[2] = {nullptr, nullptr};
    float *hacc = nullptr;
    int stage_spectra = 0;
};

namespace {

template <int NPOL> const void *pick_kernel_gather(int PPT) {
    using namespace vspec;
    switch (PPT) {
        case 1: return (const void *)fir_colfft_gather_kernel<NPOL, 1>;
        case 2: return (const void *)fir_colfft_gather_kernel<NPOL, 2>;
        case 4: return (const void *)fir_colfft_gather_kernel<NPOL, 4>;
        case 8: return (const void *)fir_colfft_gather_kernel<NPOL, 8>;
        default: return nullptr;
    }
}

template <int NPOL> const void *pick_kernel_a(int PT, int PPT) {
    using namespace vspec;
    if (PT == 1 && PPT == 1) return (const void *)fir_colfft_kernel<NPOL, 1, 1>;
    if (PT == 1 && PPT == 2) return (const void *)fir_colfft_kernel<NPOL, 1, 2>;
    if (PT == 1 && PPT == 4) return (const void *)fir_colfft_kernel<NPOL, 1, 4>;
    if (PT == 1 && PPT == 8) return (const void *)fir_colfft_kernel<NPOL, 1, 8>;
    if (PT == 2 && PPT == 1) return (const void *)fir_colfft_kernel<NPOL, 2, 1>;
    if (PT == 2 && PPT == 2) return (const void *)fir_colfft_kernel<NPOL, 2, 2>;
    if (PT == 4 && PPT == 1) return (const void *)fir_colfft_kernel<NPOL, 4, 1>;
    if (PT == 4 && PPT == 2) return (const void *)fir_colfft_kernel<NPOL, 4, 2>;
    if (PT == 8 && PPT == 1) return (const void *)fir_colfft_kernel<NPOL, 8, 1>;
    if (PT == 8 && PPT == 2) return (const void *)fir_colfft_kernel<NPOL, 8, 2>;
    if (PT == 16 && PPT == 1) return (const void *)fir_colfft_kernel<NPOL, 16, 1>;
    return nullptr;
}

// register-column kernel A for dual-pol direct FFT (2048-point tiles), N2 in
// 2 .. 256, and its column pass list (one pass up to 16 points, then 16 x N2/16)
const void *pick_kernel_coldir(int N2, size_t *smem, std::vector<int> *radices) {
    using namespace vspec;
    *radices = N2 <= 16 ? std::vector<int>{N2} : std::vector<int>{16, N2 / 16};
    switch (N2) {
        case 2: *smem = ColDir<2>::smem; return (const void *)fir_coldir_kernel<2>;
        case 4: *smem = ColDir<4>::smem; return (const void *)fir_coldir_kernel<4>;
        case 8: *smem = ColDir<8>::smem; return (const void *)fir_coldir_kernel<8>;
        case 16: *smem = ColDir<16>::smem; return (const void *)fir_coldir_kernel<16>;
        case 32: *smem = ColDir<32>::smem; return (const void *)fir_coldir_kernel<32>;
        case 64: *smem = ColDir<64>::smem; return (const void *)fir_coldir_kernel<64>;
        case 128: *smem = ColDir<128>::smem; return (const void *)fir_coldir_kernel<128>;
        case 256: *smem = ColDir<256>::smem; return (const void *)fir_coldir_kernel<256>;
    }
    return nullptr;
}

// kernel A with the column DFTs on the tensor cores (dual-pol PFB, 8 taps,
// 512-point tiles) for N2 in 16 .. 64; one column pass of radix N2 (natural order)
const void *pick_kernel_coltc(int N2, size_t *smem) {
    using namespace vspec;
    switch (N2) {
        case 16: *smem = ColTc<16>::smem; return (const void *)fir_coltc_kernel<16>;
        case 32: *smem = ColTc<32>::smem; return (const void *)fir_coltc_kernel<32>;
        case 64: *smem = ColTc<64>::smem; return (const void *)fir_coltc_kernel<64>;
    }
    return nullptr;
}

// kernel A as tensor-core products on the int8 input (pre-filter and column
// DFT together), N2 = 16 Q for Q = 1, 2, 4
// (terms = 2: high and low fp16 parts of the coefficients where they fit in
// shared memory, else 1)
const void *pick_kernel_tcfir(int N2, int P, size_t *smem, int *terms) {
    using namespace vspec;
    constexpr size_t cap = 232448 - 1024;
    switch (N2) {
        case 16: *terms = TcFir<1>::smem_for(P, 2) <= cap ? 2 : 1; *smem = TcFir<1>::smem_for(P, *terms);
                 return (const void *)fir_tcfir_kernel<1>;
        case 32: *terms = TcFir<2>::smem_for(P, 2) <= cap ? 2 : 1; *smem = TcFir<2>::smem_for(P, *terms);
                 return (const void *)fir_tcfir_kernel<2>;
        case 64: *terms = TcFir<4>::smem_for(P, 2) <= cap ? 2 : 1; *smem = TcFir<4>::smem_for(P, *terms);
                 return (const void *)fir_tcfir_kernel<4>;
    }
    return nullptr;
}

// register-column kernel A (dual-pol PFB, 8 taps, 512-point tiles) for N2 in
// 2 .. 128 and its column pass list (one pass up to 16 points, then 8 x N2/8)
const void *pick_kernel_colreg(int N2, size_t *smem, std::vector<int> *radices) {
    using namespace vspec;
    *radices = N2 <= 16 ? std::vector<int>{N2} : std::vector<int>{8, N2 / 8};
    switch (N2) {
        case 2: *smem = ColReg<2>::smem; return (const void *)fir_colreg_kernel<2>;
        case 4: *smem = ColReg<4>::smem; return (const void *)fir_colreg_kernel<4>;
        case 8: *smem = ColReg<8>::smem; return (const void *)fir_colreg_kernel<8>;
        case 16: *smem = ColReg<16>::smem; return (const void *)fir_colreg_kernel<16>;
        case 32: *smem = ColReg<32, 8>::smem; return (const void *)fir_colreg_kernel<32, 8>;
        case 64: *smem = ColReg<64, 8>::smem; return (const void *)fir_colreg_kernel<64, 8>;
        case 128: *smem = ColReg<128, 8>::smem; return (const void *)fir_colreg_kernel<128, 8>;
    }
    return nullptr;
}

constexpr int kNumKinds = 4;
const char *const kKindNames[kNumKinds] = {"fir_colfft", "rowfft_detect", "reduce", "fused_channelize"};

void release_records(vspec_plan *p) {
    for (auto &r : p->recs) {
        p->event_pool.push_back(r.start);
        p->event_pool.push_back(r.stop);
    }
    p->recs.clear();
}

cudaError_t take_event(vspec_plan *p, cudaEvent_t *ev) {
    if (!p->event_pool.empty()) {
        *ev = p->event_pool.back();
        p->event_pool.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreate(ev);
}

// Launch one kernel on st (as clusters of `cluster` CTAs if cluster > 1, as a
// cooperative launch if cluster < 0); in profiling mode bracket it with events.
vspec_status launch(vspec_plan *p, int kind, int spectra, const void *fn, dim3 grid, dim3 block,
                    void **args, size_t smem, cudaStream_t st, int cluster = 0) {
    vspec_plan *o = p->owner ? p->owner : p;  // an assist plan records into its owner
    vspec_plan::Rec r{kind, spectra, nullptr, nullptr};
    if (o->profiling) {
        VSPEC_CUDA(take_event(o, &r.start));
        VSPEC_CUDA(take_event(o, &r.stop));
        VSPEC_CUDA(cudaEventRecord(r.start, st));
    }
    cudaError_t e;
    if (cluster > 0) {
        // cluster launches go first: the highest priority places the clusters
        // before any concurrent assist CTA takes an SM they need
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = block;
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        attr[1].id = cudaLaunchAttributePriority;
        attr[1].val.priority = p->prio_high;
        cfg.attrs = attr;
        cfg.numAttrs = 2;
        e = cudaLaunchKernelExC(&cfg, fn, args);
    } else if (cluster < 0) {
        // cooperative: every CTA is resident at once (the ring kernel's CTAs wait on one another)
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = block;
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelExC(&cfg, fn, args);
    } else {
        e = cudaLaunchKernel(fn, grid, block, args, smem, st);
    }
    if (e != cudaSuccess) {
        if (o->profiling) {
            o->event_pool.push_back(r.start);
            o->event_pool.push_back(r.stop);
        }
        return cuda_fail(e, kKindNames[kind]);
    }
    if (o->profiling) {
        VSPEC_CUDA(cudaEventRecord(r.stop, st));
        o->recs.push_back(r);
    }
    return VSPEC_OK;
}

// Fold `slots` partial-sum slots of p->partial (and p->partial_comp in
// compensated plans) into d_accum: with more than 128 slots, first sum each
// group of 16 slots into its first slot, then fold the group sums.
vspec_status launch_fold(vspec_plan *p, int slots, float *d_accum, int spectra, cudaStream_t st) {
    int groups = slots, stride = 1;
    const int N = p->N, N1 = p->N1, N2 = p->N2;
    if (slots > 128) {
        groups = (slots + 15) / 16;
        stride = 16;
        const void *fold = p->npol == 2 ? (p->kahan ? (const void *)vspec::fold_slots_kernel<2, true>
                                                    : (const void *)vspec::fold_slots_kernel<2, false>)
                                        : (p->kahan ? (const void *)vspec::fold_slots_kernel<1, true>
                                                    : (const void *)vspec::fold_slots_kernel<1, false>);
        void *part = p->partial, *pcomp = p->partial_comp;
        int ns = slots, n = N;
        void *argsF[] = {&part, &pcomp, &ns, &n};
        vspec_status r = launch(p, 2, 0, fold, dim3((N + 31) / 32, groups), dim3(32, 8), argsF, 0, st);
        if (r != VSPEC_OK) return r;
    }
    const void *part = p->partial, *pcomp = p->partial_comp;
    const int *ia = p->invA, *ib = p->invB;
    void *outp = d_accum, *ocomp = p->out_comp;
    if (p->kahan) {
        void *argsR[] = {&part, &pcomp, &groups, &stride, (void *)&N, (void *)&N1, (void *)&N2, &ia, &ib, &outp, &ocomp};
        return launch(p, 2, spectra, p->kernelR, dim3((N + 31) / 32), dim3(32, 8), argsR, 0, st);
    }
    if (p->fold2048) {  // 2048-point rows, N2 >= 16: coalesced through a tile
        using namespace vspec;
        // 32 positions per CTA; for N2 < 64 8 positions and 4 slot lanes (more CTAs, shorter chains)
        const bool wide = N2 >= 64;
        const void *k = p->npol == 2 ? (wide ? (const void *)reduce2048_kernel<2, 32, 1> : (const void *)reduce2048_kernel<2, 8, 4>)
                                     : (wide ? (const void *)reduce2048_kernel<1, 32, 1> : (const void *)reduce2048_kernel<1, 8, 4>);
        void *argsT[] = {&part, &groups, &stride, (void *)&N, (void *)&N2, &ia, &outp};
        return launch(p, 2, spectra, k, dim3(N2 / 16 * 16 * (wide ? 4 : 16)), dim3(wide ? 256 : 512), argsT, 0, st);
    }
    void *argsR[] = {&part, &groups, &stride, (void *)&N, (void *)&N1, (void *)&N2, &ia, &ib, &outp};
    return launch(p, 2, spectra, p->kernelR, dim3((N + 31) / 32), dim3(32, 8), argsR, 0, st);
}

const void *pick_kernel_fused(int logn1, int pt) {
    using namespace vspec::fused;
    switch (logn1 * 100 + pt) {
        case 401: return (const void *)fused_kernel<4, 1>;
        case 408: return (const void *)fused_kernel<4, 8>;
        case 501: return (const void *)fused_kernel<5, 1>;
        case 508: return (const void *)fused_kernel<5, 8>;
        case 601: return (const void *)fused_kernel<6, 1>;
        case 608: return (const void *)fused_kernel<6, 8>;
        case 701: return (const void *)fused_kernel<7, 1>;
        case 708: return (const void *)fused_kernel<7, 8>;
        case 801: return (const void *)fused_kernel<8, 1>;
        case 808: return (const void *)fused_kernel<8, 8>;
    }
    return nullptr;
}

// Streams, events and staging buffers of vspec_execute_host.
void release_host_pipeline(vspec_plan *p) {
    if (!p->host_ready) return;
    cudaStreamDestroy(p->copy_st);
    cudaStreamDestroy(p->comp_st);
    cudaEventDestroy(p->ev_start);
    cudaEventDestroy(p->ev_done);
    for (int b = 0; b < 2; b++) {
        cudaEventDestroy(p->ev_copied[b]);
        cudaEventDestroy(p->ev_used[b]);
        cudaFree(p->stage[b]);
        p->stage[b] = nullptr;
    }
    cudaFree(p->hacc);
    p->hacc = nullptr;
    p->scratch_bytes -= p->host_bytes;
    p->host_bytes = 0;
    p->host_ready = false;
}

void free_plan(vspec_plan *p) {
    if (!p) return;
    release_records(p);
    if (p->assist) {
        free_plan(p->assist);
        cudaStreamDestroy(p->assist_st);
        cudaEventDestroy(p->ev_fork);
        cudaEventDestroy(p->ev_main);
        cudaEventDestroy(p->ev_assist);
    }
    for (cudaEvent_t e : p->event_pool) cudaEventDestroy(e);
    release_host_pipeline(p);
    cudaFree(p->coef);
    cudaFree(p->twA);
    cudaFree(p->twB);
    cudaFree(p->twZ);
    cudaFree(p->invA);
    cudaFree(p->invB);
    cudaFree(p->Z);
    cudaFree(p->partial);
    cudaFree(p->sb_scratch);
    cudaFree(p->tc_status);
    cudaFree(p->dftop);
    cudaFree(p->partial_comp);
    cudaFree(p->out_comp);
    cudaFree(p->ring_ctl);
    delete p;
}

vspec_status dev_alloc(void **ptr, size_t bytes, size_t *total) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        g_last_error = "cudaMalloc: out of memory";
        return VSPEC_ERR_OOM;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    *total += bytes;
    return VSPEC_OK;
}

// Chunk scratch: long chunks amortise the per-chunk costs (each CTA's
// partial-sum flush per row tile, the FIR window's leading frames, the ends of
// every launch); the intermediate's HBM round trip costs less than those at
// this budget (on GB300 a 1000-spectrum 32768-channel call runs at 42 GHz in
// 32 MiB chunks that stay in L2, 87 GHz in one 512 MiB chunk; a 131072-channel
// PFB call at 106 GHz in 1 GiB chunks, 111 GHz in 4 GiB ones).
// A tuned chunk may grow the scratch up to kScratchCap.
constexpr size_t kScratchBudget = 4096ull << 20;
constexpr size_t kScratchCap = 4096ull << 20;
constexpr int kMaxChunkSpectra = 8192;  // small nchan: a default chunk long enough
constexpr int kMaxWaves = 4;    // largest tuned launch, in waves of CTAs
// Ring plans: slots of about kRingSlotBytes of intermediate, partial-sum sets
// of up to kRingSetBytes, at most kRingSlotsPerLaunch slots per launch (the
// per-slot done counters).
constexpr size_t kRingSlotBytes = 32u << 20;
constexpr size_t kRingSetBytes = 16u << 20;
constexpr int kRingSlotsPerLaunch = 4096;
// Sub-band input read in place: chunks of about this much input (all bands),
// so that the bands after the first find it in L2.
constexpr size_t kSbInPlaceBytes = 32u << 20;

// Partial-sum slots a kernel-B launch of n CTAs uses: a CTA's rank among the
// CTAs that share a row tile stays below n / tiles + 2 (span_slot).
int slots_for(const vspec_plan *p, int n) { return n / (p->N2 / p->RB) + 2; }

// Partial-sum sets of a ring plan with V kernel-B tickets per row tile:
// room for a set cycle K of at least 2 (up to 64 sets in kRingSetBytes).
int ring_sets_for(const vspec_plan *p, int V) {
    const size_t per = (size_t)p->N * sizeof(float4);
    return std::max(2 * V, (int)std::min<size_t>(64, kRingSetBytes / per));
}

// Default ring shape: slots of about kRingSlotBytes (an even spectrum count),
// kernel-B tickets of 16 spectra (8 per 256-thread group), three slots with
// kernel-A work two slots ahead.
void ring_default_shape(vspec_plan *p) {
    const size_t per = (size_t)p->N * sizeof(float4);
    const int S = (int)std::min<size_t>(1024, std::max<size_t>(2, kRingSlotBytes / per)) & ~1;
    p->ringS = S;
    p->ringV = std::max(1, S / 16);
    p->ringR = 3;
    p->ringL = 2;
    p->ring_sets = ring_sets_for(p, p->ringV);
}
constexpr int kRowElems = 2048;  // target row-DFT elements per kernel-B CTA

// Fused one-pass plan: dual-pol, 2048..32768 channels, 8-tap PFB or direct.
vspec_status build_fused_plan(vspec_plan *p) {
    namespace F = vspec::fused;
    namespace W = vspec::fusedw;
    const int N = p->N;
    const int N2 = F::kN2, N1 = N / N2;
    const int logn1 = ilog2(N1);
    const int PT = p->mode == VSPEC_PFB ? 8 : 1;
    p->fused = true;
    p->fused_w = (N1 == W::kN1);  // 32768 channels: warp-local FFT variant
    p->logn1 = logn1;
    p->N1 = N1;
    p->N2 = N2;
    p->cluster = N1 / F::kCols;
    p->kernelR = (const void *)vspec::reduce_kernel<2>;
    std::vector<int> rA, rB;
    if (p->fused_w) {
        p->kernelF = PT == 8 ? (const void *)W::fused_w_kernel<8> : (const void *)W::fused_w_kernel<1>;
        p->smemF = W::smem_bytes();
        for (int i = 0; i < 3; i++) rA.push_back(W::col_radix(i));
        for (int i = 0; i < 3; i++) rB.push_back(W::row_radix(i));
    } else {
        p->kernelF = pick_kernel_fused(logn1, PT);
        p->smemF = F::smem_bytes(logn1, PT);
        for (int i = 0; i < F::kColPasses; i++) rA.push_back(F::col_radix(i));
        for (int i = 0; i < F::row_passes(logn1); i++) rB.push_back(F::row_radix(logn1, i));
    }
    int twA_n = 0, twB_n = 0;
    p->passA = make_passes(N2, rA, &twA_n);
    p->passB = make_passes(N1, rB, &twB_n);

    VSPEC_CUDA(cudaGetDevice(&p->device));
    VSPEC_CUDA(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));
    VSPEC_CUDA(raise_smem_cap(p->kernelF, p->smemF));
    if (p->cluster > 8)
        VSPEC_CUDA(cudaFuncSetAttribute(p->kernelF, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(p->cluster * std::max(1, p->num_sms / p->cluster));
        cfg.blockDim = dim3(F::kThreads);
        cfg.dynamicSmemBytes = p->smemF;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = p->cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int ncl = 0;
        VSPEC_CUDA(cudaOccupancyMaxActiveClusters(&ncl, p->kernelF, &cfg));
        if (ncl < 1) {
            g_last_error = "fused kernel: no cluster fits on this device";
            return VSPEC_ERR_UNSUPPORTED;
        }
        p->nclusters = ncl;
    }

    vspec_status st;
    size_t tot = 0;
    const int Lc = PT * N;
    if ((st = dev_alloc((void **)&p->coef, sizeof(float) * (size_t)Lc, &tot))) return st;
    if ((st = dev_alloc((void **)&p->twA, sizeof(float2) * (size_t)std::max(1, twA_n), &tot))) return st;
    if ((st = dev_alloc((void **)&p->twB, sizeof(float2) * (size_t)std::max(1, twB_n), &tot))) return st;
    if ((st = dev_alloc((void **)&p->twZ, sizeof(float2) * (size_t)N, &tot))) return st;
    if ((st = dev_alloc((void **)&p->invA, sizeof(int) * (size_t)N2, &tot))) return st;
    if ((st = dev_alloc((void **)&p->invB, sizeof(int) * (size_t)N1, &tot))) return st;
    if ((st = dev_alloc(&p->partial, (size_t)p->nclusters * N * sizeof(float4), &tot))) return st;
    p->scratch_bytes = tot;

    const std::vector<int> kA = digit_reverse(N2, rA), kB = digit_reverse(N1, rB);
    std::vector<int> invA(N2), invB(N1);
    for (int pos = 0; pos < N2; pos++) invA[kA[pos]] = pos;
    for (int pos = 0; pos < N1; pos++) invB[kB[pos]] = pos;
    int *d_kA = nullptr;
    if ((st = dev_alloc((void **)&d_kA, sizeof(int) * N2, &tot))) return st;
    cudaError_t ce = cudaMemcpy(d_kA, kA.data(), sizeof(int) * N2, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(p->invA, invA.data(), sizeof(int) * N2, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(p->invB, invB.data(), sizeof(int) * N1, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) {
        vspec::gen_coef_kernel<<<(Lc + 255) / 256, 256>>>(p->coef, N, Lc, p->mode == VSPEC_PFB ? 1 : 0, p->window);
        for (const Pass &ps : p->passA)
            if (ps.m * (ps.r - 1) > 0)
                vspec::gen_pass_tw_kernel<<<(ps.m * (ps.r - 1) + 255) / 256, 256>>>(p->twA, ps);
        for (const Pass &ps : p->passB)
            if (ps.m * (ps.r - 1) > 0)
                vspec::gen_pass_tw_kernel<<<(ps.m * (ps.r - 1) + 255) / 256, 256>>>(p->twB, ps);
        vspec::gen_twz_kernel<<<(N + 255) / 256, 256>>>(p->twZ, N, N1, N2, d_kA);
        ce = cudaGetLastError();
        if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
    }
    cudaFree(d_kA);
    if (ce != cudaSuccess) return cuda_fail(ce, "plan tables");
    return VSPEC_OK;
}

vspec_status build_plan(vspec_plan *p) {
    const int N = p->N;
    const int e = ilog2(N);
    const bool pfb = p->mode == VSPEC_PFB;
    if (!(p->flags & (VSPEC_PLAN_TWO_KERNEL | VSPEC_PLAN_TENSOR | VSPEC_PLAN_KAHAN | VSPEC_PLAN_TENSOR_INT8)) &&
        p->npol == 2 && N >= 2048 &&
        N <= 32768 && (!pfb || p->P == 8))
        return build_fused_plan(p);
    int PT = p->P <= 1 ? 1 : p->P <= 2 ? 2 : p->P <= 4 ? 4 : p->P <= 8 ? 8 : 16;
    int cmin = 32 / (2 * p->npol);  // 32-byte row segments of int8 input (one sector)
    // largest column length kernel A can hold in registers (512 threads, at
    // most 4096 points, the FIR window's registers allowing)
    auto n2max = [&]() { return PT == 1 ? 4096 / cmin : PT <= 8 ? 1024 / cmin : 512 / cmin; };
    // smallest N2 that brings N1 to at most 2048 (4096 if the columns are full)
    int N2 = 1;
    auto grow = [&]() {
        while (N / N2 > kRowElems && N2 < n2max()) N2 *= 2;
    };
    grow();
    // a PFB too long for the register FIR window reads its taps from the
    // input instead (kernel A's gather form), with direct-mode column tiles
    p->gather = pfb && N / N2 > 4096;
    if (p->gather) {
        PT = 1;
        grow();
    }
    if (p->req_n2) {  // a requested four-step split (vspec_plan_create_shaped)
        const int n2 = p->req_n2;
        const bool gather = pfb && N / n2 > 4096;
        const int cap = gather ? 4096 / cmin : n2max();
        if (!is_pow2(n2) || n2 > N || n2 > cap || N / n2 > 4096) {
            g_last_error = "requested column length outside what kernel A holds (N1 = nchan / col_len <= 4096)";
            return VSPEC_ERR_UNSUPPORTED;
        }
        N2 = n2;
        p->gather = gather;
        if (gather) PT = 1;
    }
    const int N1 = N / N2;
    if (N1 > 4096) {
        g_last_error = "nchan too large for this mode in this build";
        return VSPEC_ERR_UNSUPPORTED;
    }
    // column tile: without a FIR window in registers, enough points per CTA
    // that every thread holds eight (loads in flight); with one, the window's
    // registers allow one or two
    const int pts_target = PT == 1 ? 4096 : 512;
    int C = std::max(cmin, pts_target / N2);
    C = std::min(C, N1);
    // dual-pol direct FFT with 2048-point rows: the register-column kernel A
    // in tiles of 2048 points
    size_t smem_coldir = 0;
    std::vector<int> r_coldir;
    const void *coldir = p->npol == 2 && !pfb && N1 == 2048 && N2 >= 2 && N2 <= 256 && !p->req_cols
                             ? pick_kernel_coldir(N2, &smem_coldir, &r_coldir) : nullptr;
    if (coldir) C = 2048 / N2;
    // dual-pol PFB (5 .. 8 taps) with 2048-point rows (4096 at 2^19): the
    // register-column kernel A in 512-point tiles (for N2 = 128 rows of 4
    // samples, which the tile groups read a whole line at a time)
    const bool colreg_tiles = p->npol == 2 && pfb && PT == 8 && !p->gather && (N1 == 2048 || N1 == 4096) && N2 >= 2 &&
                              N2 <= 128 && !p->req_cols;
    if (colreg_tiles) C = 512 / N2;
    if (p->req_cols) {  // a requested tile width: the general kernel A
        const int c = p->req_cols;
        if (!is_pow2(c) || c < cmin || c > N1 || (long long)c * N2 > 4096 || N2 == 1) {
            g_last_error = "requested tile columns out of range (power of two, 32-byte rows, at most 4096 points)";
            return VSPEC_ERR_UNSUPPORTED;
        }
        C = c;
    }
    const int pts = N2 * C;
    const int TA = std::min(512, pts);
    const int PPT = pts / TA;
    p->N1 = N1;
    p->N2 = N2;
    p->C = C;
    // kernel-A blocks in groups that cover 128-byte lines of the input rows
    // together (a tile row is C samples of npol * 2 bytes)
    p->tileG = std::max(1, std::min(N1 / C, 128 / (C * p->npol * 2)));
    p->PT = PT;
    p->PPT = PPT;
    p->TA = TA;
    p->kernelA = p->gather ? (p->npol == 2 ? pick_kernel_gather<2>(PPT) : pick_kernel_gather<1>(PPT))
                           : (p->npol == 2 ? pick_kernel_a<2>(PT, PPT) : pick_kernel_a<1>(PT, PPT));
    if (coldir) {
        p->kernelA = coldir;
        p->formA = "coldir";
    }
    if (p->gather) p->formA = "gather";
    if (!p->kernelA) {
        g_last_error = "no kernel instance for this tap count and size";
        return VSPEC_ERR_UNSUPPORTED;
    }
    // a one-row transform (N2 == 1) needs no column pass: kernel B applies the
    // FIR to the int8 input in its first pass, and there is no chunk scratch
    p->fir_b = N2 == 1 && !(p->flags & VSPEC_PLAN_TENSOR);
    p->kernelB = p->npol == 2 ? (p->fir_b ? (const void *)vspec::rowfft_detect_kernel<2, false, true>
                                          : (const void *)vspec::rowfft_detect_kernel<2>)
                              : (p->fir_b ? (const void *)vspec::rowfft_detect_kernel<1, false, true>
                                          : (const void *)vspec::rowfft_detect_kernel<1>);
    p->kernelR = p->npol == 2 ? (const void *)vspec::reduce_kernel<2> : (const void *)vspec::reduce_kernel<1>;

    const int e2 = ilog2(N2), e1 = e - e2;
    // Kernel A keeps its register window live through the column DFTs: cap
    // the butterfly width so both fit in 128 registers.
    const int capA = vspec::col_radix_cap(p->npol, PT, PPT);
    const int maxbitsA = capA == 16 ? 4 : capA == 8 ? 3 : 2;
    // dual-pol PFB (5 .. 8 taps) with columns of 2 .. 128 points in 512-point
    // tiles: the register-column kernel A and its own column pass list
    size_t smem_colreg = 0;
    std::vector<int> r_colreg;
    const void *colreg = p->npol == 2 && pfb && PT == 8 && PPT == 1 && !p->gather && N2 * C == 512 && !p->req_cols
                             ? pick_kernel_colreg(N2, &smem_colreg, &r_colreg) : nullptr;
    if (colreg) {
        p->kernelA = colreg;
        p->formA = "colreg";
    }
    // tensor-core plans with 2048-point rows and N2 = 16, 32, 64:
    //  - VSPEC_PLAN_TENSOR_INT8 (PFB of at most 8 taps, or direct): pre-filter
    //    and column DFT as one tensor-core product on the int8 input, one
    //    column per CTA, groups of 8 CTAs on 8 adjacent columns;
    //  - VSPEC_PLAN_TENSOR, dual-pol PFB of 5 .. 8 taps: the register-column
    //    FIR, then the column DFTs as tensor-core products (fp16 Y, split F).
    size_t smem_tcA = 0;
    const bool want_int8 = (p->flags & VSPEC_PLAN_TENSOR_INT8) != 0;
    const void *tcfir = want_int8 && p->npol == 2 && N1 == 2048 && p->P <= 8 && !p->gather
                            ? pick_kernel_tcfir(N2, p->P, &smem_tcA, &p->bterms) : nullptr;
    if (want_int8 && !tcfir) {
        g_last_error = "the int8 tensor-core form needs dual-pol, at most 8 taps and nchan 2^15 .. 2^17";
        return VSPEC_ERR_UNSUPPORTED;
    }
    const void *coltc = !want_int8 && (p->flags & VSPEC_PLAN_TENSOR) && colreg && N1 == 2048
                            ? pick_kernel_coltc(N2, &smem_tcA) : nullptr;
    if (tcfir) {
        p->kernelA = tcfir;
        p->formA = "tensor-int8";
        p->tc_cols = p->tc_int8 = true;
        p->C = 1;
        p->tileG = 8;
        p->TA = 512;
        p->PPT = 1;
    }
    if (coltc) {
        p->kernelA = coltc;
        p->formA = "tensor";
        p->tc_cols = true;
    }
    if (p->fir_b) p->formA = "none";
    // dual-pol 4096-point rows without a pre-filter in kernel B, compensated
    // sums or tensor-core rows: four radix-8 passes (row4096_kernel)
    const bool row4096 = N1 == 4096 && p->npol == 2 && !p->fir_b &&
                         !(p->flags & (VSPEC_PLAN_KAHAN | VSPEC_PLAN_TENSOR | VSPEC_PLAN_TENSOR_INT8));
    const std::vector<int> rA = (tcfir || coltc) ? std::vector<int>{N2} : colreg ? r_colreg : coldir ? r_coldir
                                                                               : radix_list(e2, maxbitsA),
                           rB = row4096 ? std::vector<int>{8, 8, 8, 8} : radix_list(e1);
    int twA_n = 0, twB_n = 0;
    p->passA = make_passes(N2, rA, &twA_n);
    p->passB = make_passes(N1, rB, &twB_n);
    if ((int)p->passA.size() > vspec::kMaxPasses || (int)p->passB.size() > vspec::kMaxPasses ||
        p->passB.empty()) {
        g_last_error = "pass count out of range";
        return VSPEC_ERR_UNSUPPORTED;
    }
    p->RB = std::max(1, std::min(N2, kRowElems / N1));
    int maxb = 1;
    for (const Pass &ps : p->passB) maxb = std::max(maxb, p->RB * (N1 / ps.r));
    p->TB = std::min(256, std::max(32, maxb));
    if ((p->flags & VSPEC_PLAN_TENSOR) && !p->tc_cols) {
        if (p->npol != 2 || N1 != vspec::kTcN1 || p->RB != 1 || p->passB[0].r != 16) {
            g_last_error = "tensor-core stage needs dual-pol and 2048-point rows (nchan 2^11 .. 2^20)";
            return VSPEC_ERR_UNSUPPORTED;
        }
        p->tc = true;
        p->formB = "tensor";
        p->kernelB = (p->flags & VSPEC_PLAN_KAHAN) ? (const void *)vspec::rowfft_detect_tc_kernel<3, true>
                                                   : (const void *)vspec::rowfft_detect_tc_kernel<3, false>;
        p->TB = 256;
    }
    if (p->flags & VSPEC_PLAN_KAHAN) {
        p->kahan = true;
        if (!p->tc)
            p->kernelB = p->npol == 2 ? (p->fir_b ? (const void *)vspec::rowfft_detect_kernel<2, true, true>
                                                  : (const void *)vspec::rowfft_detect_kernel<2, true>)
                                      : (p->fir_b ? (const void *)vspec::rowfft_detect_kernel<1, true, true>
                                                  : (const void *)vspec::rowfft_detect_kernel<1, true>);
        p->kernelR = p->npol == 2 ? (const void *)vspec::reduce_kahan_kernel<2>
                                  : (const void *)vspec::reduce_kahan_kernel<1>;
    }

    const size_t elem = p->npol == 2 ? sizeof(float4) : sizeof(float2);
    const size_t accel = p->npol == 2 ? sizeof(float4) : sizeof(float);
    // data [PT][N2][C], twiddle tile [N2][C], two batches of raw frames
    p->smemA = (size_t)PT * N2 * C * elem + (size_t)N2 * C * sizeof(float2) +
               (!p->gather ? 2 * (size_t)PT * N2 * C * p->npol * 2 : 0);
    if (colreg) p->smemA = smem_colreg;
    if (tcfir || coltc) p->smemA = smem_tcA;
    if (coldir) p->smemA = smem_coldir;
    p->smemB = (size_t)p->RB * (N1 + (N1 >> 4)) * elem + (size_t)p->RB * N1 * accel;
    if (p->kahan) p->smemB += (size_t)p->RB * N1 * accel;
    if (p->fir_b)  // one-row transform: frame ring and coefficients (general row kernel)
        p->smemB = (p->npol == 2 ? (p->kahan ? vspec::row_ring_offset<2, true>(p->RB, N1)
                                             : vspec::row_ring_offset<2, false>(p->RB, N1))
                                 : (p->kahan ? vspec::row_ring_offset<1, true>(p->RB, N1)
                                             : vspec::row_ring_offset<1, false>(p->RB, N1))) +
                   vspec::row_ring_bytes(p->npol, p->P, N1);
    if (p->tc) p->smemB = vspec::tc_rowfft_smem(p->kahan);
    // 2048-point rows (radix 16, 16, 8): the paired-spectra row kernel with
    // register accumulators
    if (!p->tc && N1 == 2048 && p->RB == 1 && p->passB.size() == 3 && p->passB[0].r == 16 &&
        p->passB[1].r == 16 && p->passB[2].r == 8) {
        using namespace vspec;
        const bool k = p->kahan, f = p->fir_b;
        if (p->npol == 2 && coltc)  // scratch elements in the tensor-core column kernel's order
            p->kernelB = k ? (const void *)row2048_kernel<2, true, false, true> : (const void *)row2048_kernel<2, false, false, true>;
        else if (p->npol == 2)
            p->kernelB = k ? (f ? (const void *)row2048_kernel<2, true, true> : (const void *)row2048_kernel<2, true, false>)
                           : (f ? (const void *)row2048_kernel<2, false, true> : (const void *)row2048_kernel<2, false, false>);
        else
            p->kernelB = k ? (f ? (const void *)row2048_kernel<1, true, true> : (const void *)row2048_kernel<1, true, false>)
                           : (f ? (const void *)row2048_kernel<1, false, true> : (const void *)row2048_kernel<1, false, false>);
        p->TB = 256;
        p->smemB = 2 * (size_t)kRow2048Stride * elem;
        p->formB = "row2048";
        p->fold2048 = N2 >= 16 && !p->kahan;
    }
    // 4096-point rows (radix 8, 8, 8, 8): one spectrum per pass sequence,
    // register accumulators
    if (row4096 && !p->tc && p->RB == 1 && p->passB.size() == 4) {
        p->kernelB = (const void *)vspec::row4096_kernel<false>;
        p->TB = 512;
        p->smemB = (size_t)vspec::kRow4096Stride * elem;
        p->formB = "row4096";
    }

    // the persistent ring form: the register-column kernel A and the paired
    // 2048-point row kernel as tickets of one launch
    if (p->flags & VSPEC_PLAN_RING) {
        if (!colreg || std::strcmp(p->formB, "row2048") != 0 || p->npol != 2 || p->kahan || p->tc || p->fir_b) {
            g_last_error = "the ring form needs dual-pol PFB of 5..8 taps with 2048-point rows (nchan 2^12..2^18)";
            return VSPEC_ERR_UNSUPPORTED;
        }
        p->kernelRing = vspec_pick_kernel_ring(N2, &p->smemRing);
        if (!p->kernelRing) {
            g_last_error = "no ring kernel instance for this column length";
            return VSPEC_ERR_UNSUPPORTED;
        }
        p->ring = true;
    }

    VSPEC_CUDA(cudaGetDevice(&p->device));
    VSPEC_CUDA(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));
    if (p->ring) {
        int coop = 0, occ = 0;
        VSPEC_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, p->device));
        VSPEC_CUDA(raise_smem_cap(p->kernelRing, p->smemRing));
        VSPEC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, p->kernelRing, 512, p->smemRing));
        if (!coop || occ < 1) {
            g_last_error = "the ring kernel needs cooperative launches and one resident CTA per SM";
            return VSPEC_ERR_UNSUPPORTED;
        }
        p->ring_grid = p->num_sms * occ;
    }
    VSPEC_CUDA(raise_smem_cap(p->kernelA, p->smemA));
    VSPEC_CUDA(raise_smem_cap(p->kernelB, p->smemB));
    VSPEC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p->occA, p->kernelA, p->TA, p->smemA));
    VSPEC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p->occB, p->kernelB, p->TB, p->smemB));
    if (p->occA < 1 || p->occB < 1) {
        g_last_error = "kernel does not fit on an SM";
        return VSPEC_ERR_UNSUPPORTED;
    }

    const size_t per_spec = (size_t)N * elem;
    p->sc_cap = (int)std::max<size_t>(1, kScratchCap / per_spec);
    p->sc_max = std::min({p->sc_cap, kMaxChunkSpectra, (int)std::max<size_t>(1, kScratchBudget / per_spec)});
    if (p->fir_b) p->sc_cap = p->sc_max = kMaxChunkSpectra;  // launch length only: no scratch
    // partial-sum slots for the largest kernel-B launch a tuning may ask for
    p->slots_cap = slots_for(p, kMaxWaves * p->num_sms * p->occB);

    // device tables and scratch
    vspec_status st;
    size_t tot = 0;
    const int Lc = (pfb ? p->P : 1) * N;
    if ((st = dev_alloc((void **)&p->coef, sizeof(float) * (size_t)Lc, &tot))) return st;
    if ((st = dev_alloc((void **)&p->twA, sizeof(float2) * (size_t)std::max(1, twA_n), &tot))) return st;
    if ((st = dev_alloc((void **)&p->twB, sizeof(float2) * (size_t)std::max(1, twB_n), &tot))) return st;
    if ((st = dev_alloc((void **)&p->twZ, sizeof(float2) * (size_t)N, &tot))) return st;
    if ((st = dev_alloc((void **)&p->invA, sizeof(int) * (size_t)N2, &tot))) return st;
    if ((st = dev_alloc((void **)&p->invB, sizeof(int) * (size_t)N1, &tot))) return st;
    p->sc_alloc = p->fir_b ? 0 : p->sc_max;
    if (p->ring) {  // the ring and its partial-sum sets instead of the chunk scratch
        ring_default_shape(p);
        p->sc_alloc = p->sc_max = p->sc_cap = p->ringR * p->ringS;
        p->slots_cap = p->ring_sets;
        if ((st = dev_alloc((void **)&p->ring_ctl, sizeof(int) * (2 + 2 * (size_t)kRingSlotsPerLaunch), &tot)))
            return st;
    }
    if ((st = dev_alloc(&p->Z, (size_t)std::max(1, p->sc_alloc) * N * elem, &tot))) return st;
    if ((st = dev_alloc(&p->partial, (size_t)p->slots_cap * N * accel, &tot))) return st;
    if (p->tc || p->tc_cols || p->ring) {
        if ((st = dev_alloc((void **)&p->tc_status, sizeof(int), &tot))) return st;
        VSPEC_CUDA(cudaMemset(p->tc_status, 0, sizeof(int)));
    }
    if (p->tc_int8) {  // the per-column B blocks: N1 columns x Q residues x P taps x 2 KiB (x terms)
        if ((st = dev_alloc((void **)&p->dftop, (size_t)N1 * (N2 / 16) * p->P * p->bterms * 2048, &tot)))
            return st;
    } else if (p->tc_cols) {  // the column DFT operand F, hi and lo, then the scaled four-step twiddles
        if ((st = dev_alloc((void **)&p->dftop, (size_t)2 * (2 * N2) * (2 * N2) * 2 + (size_t)N * sizeof(float2),
                            &tot)))
            return st;
    }
    if (p->kahan) {
        if ((st = dev_alloc(&p->partial_comp, (size_t)p->slots_cap * N * accel, &tot))) return st;
        if ((st = dev_alloc(&p->out_comp, (size_t)N * accel, &tot))) return st;
        VSPEC_CUDA(cudaMemset(p->out_comp, 0, (size_t)N * accel));
    }
    p->scratch_bytes = tot;

    // digit-reversal maps (host) -> inverse maps for the final scatter
    const std::vector<int> kA = digit_reverse(N2, rA), kB = digit_reverse(N1, rB);
    std::vector<int> invA(N2), invB(N1);
    for (int pos = 0; pos < N2; pos++) invA[kA[pos]] = pos;
    for (int pos = 0; pos < N1; pos++) invB[kB[pos]] = pos;
    int *d_kA = nullptr;
    if ((st = dev_alloc((void **)&d_kA, sizeof(int) * N2, &tot))) return st;
    p->scratch_bytes = tot - sizeof(int) * N2;
    cudaStream_t s0 = nullptr;
    cudaError_t ce = cudaMemcpy(d_kA, kA.data(), sizeof(int) * N2, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(p->invA, invA.data(), sizeof(int) * N2, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(p->invB, invB.data(), sizeof(int) * N1, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) {
        vspec::gen_coef_kernel<<<(Lc + 255) / 256, 256, 0, s0>>>(p->coef, N, Lc, pfb ? 1 : 0, p->window);
        for (const Pass &ps : p->passA)
            if (ps.m * (ps.r - 1) > 0)
                vspec::gen_pass_tw_kernel<<<(ps.m * (ps.r - 1) + 255) / 256, 256, 0, s0>>>(p->twA, ps);
        for (const Pass &ps : p->passB)
            if (ps.m * (ps.r - 1) > 0)
                vspec::gen_pass_tw_kernel<<<(ps.m * (ps.r - 1) + 255) / 256, 256, 0, s0>>>(p->twB, ps);
        vspec::gen_twz_kernel<<<(N + 255) / 256, 256, 0, s0>>>(p->twZ, N, N1, N2, d_kA);
        if (p->tc_cols && !p->tc_int8) {
            vspec::gen_coltc_operand_kernel<<<(4 * N2 * N2 + 255) / 256, 256, 0, s0>>>(p->dftop, N2);
            vspec::gen_coltc_twz_kernel<<<(N + 255) / 256, 256, 0, s0>>>(
                reinterpret_cast<float2 *>(p->dftop + (size_t)2 * (2 * N2) * (2 * N2) * 2), p->twZ, N, N1, N2);
        }
        if (p->tc_int8) {
            const long long nb = (long long)N1 * (N2 / 16) * p->P * 1024;
            vspec::gen_tcfir_operand_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, s0>>>(p->dftop, p->coef, N, N1,
                                                                                      N2 / 16, p->P, p->bterms);
        }
        ce = cudaGetLastError();
        if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
    }
    cudaFree(d_kA);
    if (ce != cudaSuccess) return cuda_fail(ce, "plan tables");
    return VSPEC_OK;
}

bool aligned16(const void *ptr) { return ((uintptr_t)ptr & 15u) == 0; }

}  // namespace

extern "C" {

const char *vspec_status_string(vspec_status s) {
    switch (s) {
        case VSPEC_OK: return "ok";
        case VSPEC_ERR_INVALID_ARG: return "invalid argument";
        case VSPEC_ERR_UNSUPPORTED: return "unsupported configuration";
        case VSPEC_ERR_ALIGNMENT: return "pointer not 16-byte aligned";
        case VSPEC_ERR_CUDA: return "CUDA error";
        case VSPEC_ERR_OOM: return "out of device memory";
        case VSPEC_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    }
    return "unknown status";
}

const char *vspec_last_error(void) { return g_last_error.c_str(); }

vspec_status vspec_plan_create(vspec_plan **out, int nchan, int ntaps, int npol, vspec_mode mode,
                               vspec_window window) {
    return vspec_plan_create_ex(out, nchan, ntaps, npol, mode, window, 0u);
}

// Fused plans own a two-kernel plan of the same problem, for two uses.
// (1) Long calls: the two-kernel path spreads its work evenly over every SM
// and hides its memory latency better, and beyond a per-size number of
// spectra it is the faster path; below it the fused kernel's smaller fixed
// cost wins. The thresholds come from measurements on GB300 (both paths
// timed at 50 to 4000 spectra per call); at 2048 channels the fused path is
// faster at every length.
// (2) Assist: on a device whose SM count is not a multiple of the cluster
// size, the two-kernel plan can channelize a share of a call's spectra on
// the SMs the clusters leave idle, concurrently with the fused kernel. The
// default share balances the two finishing times: idle SMs at the two-kernel
// path's per-SM rate against the clusters' SMs at the fused kernel's (about
// 0.62 of it with an 8-tap PFB, 0.70 in direct mode). With only a few idle
// SMs the second path's fixed cost outweighs them.
constexpr int kTwoKernelFrom[2][5] = {
    {INT_MAX, 800, 300, 100, 0},  // PFB, nchan 2048 .. 32768
    {INT_MAX, 900, 300, 100, 70}  // direct
};
constexpr double kAssistPerSmRate = 0.62;        // PFB
constexpr double kAssistPerSmRateDirect = 0.70;  // direct FFT
constexpr int kAssistMinSms = 24;      // fewer idle SMs: no assist
constexpr int kAssistMinSpectra = 32;  // smallest share worth a second path
constexpr int kAssistMaxPermille = 900;

static vspec_status setup_assist(vspec_plan *p) {
    VSPEC_CUDA(cudaDeviceGetStreamPriorityRange(nullptr, &p->prio_high));
    const int busy = p->cluster * p->nclusters;
    const int idle = p->num_sms - busy;
    const int lg = ilog2(p->N) - 11;
    p->two_kernel_from = (lg >= 0 && lg < 5) ? kTwoKernelFrom[p->mode == VSPEC_PFB ? 0 : 1][lg] : INT_MAX;
    if (idle < kAssistMinSms && p->two_kernel_from == INT_MAX) return VSPEC_OK;
    vspec_plan *a = nullptr;
    vspec_status st = vspec_plan_create_ex(&a, p->N, p->mode == VSPEC_PFB ? p->P : 1, p->npol,
                                           (vspec_mode)p->mode, (vspec_window)p->window, VSPEC_PLAN_TWO_KERNEL);
    if (st != VSPEC_OK) return st;
    a->owner = p;
    p->assist = a;
    p->scratch_bytes += a->scratch_bytes;
    if (idle >= kAssistMinSms) {
        const double w = idle * (p->mode == VSPEC_PFB ? kAssistPerSmRate : kAssistPerSmRateDirect);
        p->assist_permille = (int)(1000.0 * w / (w + busy) + 0.5);
    }
    VSPEC_CUDA(cudaStreamCreateWithFlags(&p->assist_st, cudaStreamNonBlocking));
    VSPEC_CUDA(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
    VSPEC_CUDA(cudaEventCreateWithFlags(&p->ev_main, cudaEventDisableTiming));
    VSPEC_CUDA(cudaEventCreateWithFlags(&p->ev_assist, cudaEventDisableTiming));
    return VSPEC_OK;
}

vspec_status vspec_plan_create_ex(vspec_plan **out, int nchan, int ntaps, int npol, vspec_mode mode,
                                  vspec_window window, unsigned flags) {
    return vspec_plan_create_shaped(out, nchan, ntaps, npol, mode, window, flags, 0, 0);
}

vspec_status vspec_plan_get_shape(const vspec_plan *plan, int *col_len, int *tile_cols) {
    if (!plan) return VSPEC_ERR_INVALID_ARG;
    const vspec_plan *t = plan->fused && plan->assist ? plan->assist : plan;
    if (col_len) *col_len = plan->fused && !plan->assist ? 0 : t->N2;
    if (tile_cols) *tile_cols = plan->fused && !plan->assist ? 0 : t->C;
    return VSPEC_OK;
}

vspec_status vspec_plan_create_shaped(vspec_plan **out, int nchan, int ntaps, int npol, vspec_mode mode,
                                      vspec_window window, unsigned flags, int col_len, int tile_cols) {
    if (!out) return VSPEC_ERR_INVALID_ARG;
    if (col_len < 0 || tile_cols < 0) {
        *out = nullptr;
        return VSPEC_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!is_pow2(nchan) || nchan < 16 || nchan > (1 << 20)) return VSPEC_ERR_INVALID_ARG;
    if (npol != 1 && npol != 2) return VSPEC_ERR_INVALID_ARG;
    if (mode != VSPEC_PFB && mode != VSPEC_DIRECT) return VSPEC_ERR_INVALID_ARG;
    if (window != VSPEC_WIN_RECT && window != VSPEC_WIN_HANN && window != VSPEC_WIN_HAMMING)
        return VSPEC_ERR_INVALID_ARG;
    if (mode == VSPEC_PFB && (ntaps < 1 || ntaps > 16)) return VSPEC_ERR_INVALID_ARG;
    if (mode == VSPEC_DIRECT && (ntaps < 0 || ntaps > 1)) return VSPEC_ERR_INVALID_ARG;

    vspec_plan *p = new (std::nothrow) vspec_plan();
    if (!p) return VSPEC_ERR_OOM;
    p->N = nchan;
    p->P = mode == VSPEC_PFB ? ntaps : 1;
    p->npol = npol;
    p->mode = mode;
    p->window = window;
    if (flags & ~(unsigned)(VSPEC_PLAN_TWO_KERNEL | VSPEC_PLAN_TENSOR | VSPEC_PLAN_KAHAN | VSPEC_PLAN_TENSOR_INT8 |
                            VSPEC_PLAN_RING)) {
        delete p;
        *out = nullptr;
        return VSPEC_ERR_INVALID_ARG;
    }
    p->flags = flags;
    p->req_n2 = col_len;
    p->req_cols = tile_cols;
    if (col_len || tile_cols) p->flags |= VSPEC_PLAN_TWO_KERNEL;  // a shape is a two-kernel shape
    if (flags & VSPEC_PLAN_RING) p->flags |= VSPEC_PLAN_TWO_KERNEL;  // the ring runs kernels A and B
    vspec_status st = build_plan(p);
    if (st == VSPEC_OK && p->fused) st = setup_assist(p);
    if (st != VSPEC_OK) {
        free_plan(p);
        return st;
    }
    *out = p;
    return VSPEC_OK;
}

static bool sb_in_place(const vspec_plan *p, int nsub);
static vspec_plan *sb_plan(vspec_plan *p);

vspec_status vspec_plan_create_sb(vspec_plan **out, int nchan, int ntaps, int npol, int nsub,
                                  vspec_mode mode, vspec_window window, unsigned flags) {
    if (!out) return VSPEC_ERR_INVALID_ARG;
    *out = nullptr;
    if (nsub < 1 || nsub > 16) return VSPEC_ERR_INVALID_ARG;
    if (nsub > 1 && (flags & VSPEC_PLAN_KAHAN)) {
        g_last_error = "compensated accumulation is not available in sub-band modes";
        return VSPEC_ERR_UNSUPPORTED;
    }
    vspec_status st = vspec_plan_create_ex(out, nchan, ntaps, npol, mode, window, flags);
    if (st != VSPEC_OK || nsub == 1) return st;
    vspec_plan *p = *out;
    p->nsub = nsub;
    if (sb_in_place(sb_plan(p), nsub)) return VSPEC_OK;  // kernel A reads each band in place: no de-interleave scratch
    const int Peff = mode == VSPEC_PFB ? ntaps : 1;
    const size_t per_spec = (size_t)nchan * npol * 2;  // bytes of one sub-band per spectrum
    p->sb_chunk = (int)std::max<size_t>(1, (64u << 20) / (per_spec * nsub));
    size_t tot = 0;
    st = dev_alloc((void **)&p->sb_scratch, (size_t)nsub * (p->sb_chunk + Peff - 1) * per_spec, &tot);
    if (st != VSPEC_OK) {
        free_plan(p);
        *out = nullptr;
        return st;
    }
    p->scratch_bytes += tot;
    return VSPEC_OK;
}

vspec_status vspec_plan_destroy(vspec_plan *plan) {
    free_plan(plan);
    return VSPEC_OK;
}

vspec_status vspec_plan_info(const vspec_plan *plan, size_t *scratch_bytes, int *hbm_passes) {
    if (!plan) return VSPEC_ERR_INVALID_ARG;
    if (scratch_bytes) *scratch_bytes = plan->scratch_bytes;
    if (hbm_passes) {
        // the input is read once; the two-kernel path's chunk scratch adds a
        // write and a read of the intermediate when it cannot stay in L2
        int l2 = 0;
        if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, plan->device) != cudaSuccess) l2 = 0;
        // (a fused plan reports the two-kernel path it switches to on long calls)
        const vspec_plan *tk = !plan->fused ? plan : plan->two_kernel_from < INT_MAX ? plan->assist : nullptr;
        const size_t zb = tk ? (size_t)tk->sc_max * tk->N * (tk->npol == 2 ? sizeof(float4) : sizeof(float2)) : 0;
        *hbm_passes = (tk && !tk->fir_b && !tk->ring && zb > (size_t)l2 / 2) ? 2 : 1;
    }
    return VSPEC_OK;
}

vspec_status vspec_plan_describe(const vspec_plan *plan, char *buf, size_t len) {
    if (!plan || !buf || len == 0) return VSPEC_ERR_INVALID_ARG;
    auto two_kernel = [](const vspec_plan *t) {
        std::string d = "two-kernel N1=" + std::to_string(t->N1) + " N2=" + std::to_string(t->N2) +
                        " C=" + std::to_string(t->C) + " A=" + t->formA + " B=" + t->formB +
                        " chunk=" + std::to_string(t->sc_max);
        if (t->fir_b) d += " fir-in-B";
        if (t->kahan) d += " kahan";
        if (t->ring)
            d += " ring S=" + std::to_string(t->ringS) + " R=" + std::to_string(t->ringR) + " L=" +
                 std::to_string(t->ringL) + " V=" + std::to_string(t->ringV);
        return d;
    };
    std::string d;
    if (plan->fused) {
        d = "fused K=" + std::to_string(plan->cluster);
        if (plan->assist) d += " | " + two_kernel(plan->assist);
    } else {
        d = two_kernel(plan);
    }
    const size_t n = std::min(len - 1, d.size());
    std::memcpy(buf, d.data(), n);
    buf[n] = '\0';
    return VSPEC_OK;
}

vspec_status vspec_plan_get_tuning(const vspec_plan *plan, vspec_tuning *current, vspec_tuning *limit) {
    if (!plan) return VSPEC_ERR_INVALID_ARG;
    const vspec_plan *tk = plan->fused ? plan->assist : plan;  // the plan that runs the two-kernel path
    vspec_tuning cur{0, 0, 0, 0, plan->fused ? plan->two_kernel_from : 0};
    vspec_tuning lim{0, 0, 0, 0, plan->fused && plan->assist ? INT_MAX : cur.two_kernel_from};
    if (tk) {
        cur.chunk_spectra = tk->sc_max;
        cur.blocks_a = tk->blocks_a;
        cur.blocks_b = tk->blocks_b;
        lim.chunk_spectra = tk->sc_cap;
        lim.blocks_a = kMaxWaves * tk->num_sms * tk->occA;
        lim.blocks_b = kMaxWaves * tk->num_sms * tk->occB;
    }
    if (plan->fused) {
        const bool can_assist = plan->assist && plan->num_sms - plan->cluster * plan->nclusters >= kAssistMinSms;
        cur.assist_permille = can_assist ? plan->assist_permille : 0;
        lim.assist_permille = can_assist ? kAssistMaxPermille : 0;
    }
    if (current) *current = cur;
    if (limit) *limit = lim;
    return VSPEC_OK;
}

vspec_status vspec_plan_set_tuning(vspec_plan *plan, const vspec_tuning *t) {
    if (!plan || !t) return VSPEC_ERR_INVALID_ARG;
    if (plan->ring) {
        g_last_error = "a ring plan is shaped by vspec_plan_set_ring";
        return VSPEC_ERR_UNSUPPORTED;
    }
    vspec_tuning lim{};
    vspec_plan_get_tuning(plan, nullptr, &lim);
    vspec_plan *tk = plan->fused ? plan->assist : plan;
    const bool chunk_ok = tk ? (t->chunk_spectra >= 1 && t->chunk_spectra <= lim.chunk_spectra)
                             : t->chunk_spectra == 0;
    const bool two_kernel_ok = plan->fused ? (plan->assist ? t->two_kernel_from >= 0 : t->two_kernel_from == INT_MAX)
                                           : t->two_kernel_from == 0;
    if (!chunk_ok || t->blocks_a < 0 || t->blocks_a > lim.blocks_a || t->blocks_b < 0 ||
        t->blocks_b > lim.blocks_b || t->assist_permille < 0 || t->assist_permille > lim.assist_permille ||
        !two_kernel_ok) {
        g_last_error = "tuning value out of range for this plan";
        return VSPEC_ERR_INVALID_ARG;
    }
    if (tk) {
        if (!tk->fir_b && t->chunk_spectra > tk->sc_alloc) {  // grow the chunk scratch
            const size_t elem = tk->npol == 2 ? sizeof(float4) : sizeof(float2);
            const size_t old_bytes = (size_t)tk->sc_alloc * tk->N * elem;
            void *z = nullptr;
            size_t tot = 0;
            VSPEC_CUDA(cudaDeviceSynchronize());
            vspec_status st = dev_alloc(&z, (size_t)t->chunk_spectra * tk->N * elem, &tot);
            if (st != VSPEC_OK) return st;
            cudaFree(tk->Z);
            tk->Z = z;
            tk->scratch_bytes += tot - old_bytes;
            if (tk != plan) plan->scratch_bytes += tot - old_bytes;
            tk->sc_alloc = t->chunk_spectra;
        }
        tk->sc_max = t->chunk_spectra;
        tk->blocks_a = t->blocks_a;
        tk->blocks_b = t->blocks_b;
    }
    if (plan->fused) {
        plan->assist_permille = t->assist_permille;
        plan->two_kernel_from = t->two_kernel_from;
    }
    return VSPEC_OK;
}

vspec_status vspec_plan_set_ring(vspec_plan *plan, int slot_spectra, int ring_slots, int lookahead, int row_parts) {
    if (!plan) return VSPEC_ERR_INVALID_ARG;
    if (!plan->ring) {
        g_last_error = "not a ring plan (VSPEC_PLAN_RING)";
        return VSPEC_ERR_UNSUPPORTED;
    }
    if (slot_spectra < 0 || ring_slots < 0 || lookahead < 0 || row_parts < 0) return VSPEC_ERR_INVALID_ARG;
    const int S = slot_spectra ? slot_spectra : plan->ringS;
    const int R = ring_slots ? ring_slots : plan->ringR;
    const int L = lookahead ? lookahead : plan->ringL;
    const int V = row_parts ? row_parts : (slot_spectra ? std::max(1, S / 16) : plan->ringV);
    if (S < 2 || S > 1024 || (S & 1) || R < 1 || R > 16 || L < 1 || L > 15 || R < L || V < 1 || S % V ||
        ((S / V) & 1) || S / V > 32) {
        g_last_error = "ring shape out of range";
        return VSPEC_ERR_INVALID_ARG;
    }
    const size_t elem = sizeof(float4);
    const int sets = ring_sets_for(plan, V);
    VSPEC_CUDA(cudaDeviceSynchronize());
    cudaFree(plan->Z);
    cudaFree(plan->partial);
    plan->Z = plan->partial = nullptr;
    plan->scratch_bytes -= (size_t)plan->sc_alloc * plan->N * elem + (size_t)plan->slots_cap * plan->N * elem;
    plan->sc_alloc = plan->sc_max = plan->sc_cap = 0;
    plan->slots_cap = 0;
    size_t tot = 0;
    vspec_status st = dev_alloc(&plan->Z, (size_t)R * S * plan->N * elem, &tot);
    if (st == VSPEC_OK) st = dev_alloc(&plan->partial, (size_t)sets * plan->N * elem, &tot);
    if (st != VSPEC_OK) {  // the plan keeps no ring: a later call fails until a shape fits
        cudaFree(plan->Z);
        plan->Z = nullptr;
        plan->ringS = 0;
        return st;
    }
    plan->scratch_bytes += tot;
    plan->ringS = S;
    plan->ringR = R;
    plan->ringL = L;
    plan->ringV = V;
    plan->ring_sets = sets;
    plan->sc_alloc = plan->sc_max = plan->sc_cap = R * S;
    plan->slots_cap = sets;
    return VSPEC_OK;
}

vspec_status vspec_plan_get_ring(const vspec_plan *plan, int *slot_spectra, int *ring_slots, int *lookahead,
                                 int *row_parts) {
    if (!plan) return VSPEC_ERR_INVALID_ARG;
    if (!plan->ring) {
        g_last_error = "not a ring plan (VSPEC_PLAN_RING)";
        return VSPEC_ERR_UNSUPPORTED;
    }
    if (slot_spectra) *slot_spectra = plan->ringS;
    if (ring_slots) *ring_slots = plan->ringR;
    if (lookahead) *lookahead = plan->ringL;
    if (row_parts) *row_parts = plan->ringV;
    return VSPEC_OK;
}

vspec_status vspec_plan_trim_scratch(vspec_plan *plan) {
    if (!plan) return VSPEC_ERR_INVALID_ARG;
    vspec_plan *tk = plan->fused ? plan->assist : plan;
    if (!tk || tk->fir_b || tk->sc_alloc <= tk->sc_max) return VSPEC_OK;
    const size_t elem = tk->npol == 2 ? sizeof(float4) : sizeof(float2);
    const size_t old_bytes = (size_t)tk->sc_alloc * tk->N * elem;
    VSPEC_CUDA(cudaDeviceSynchronize());
    cudaFree(tk->Z);
    tk->Z = nullptr;
    size_t tot = 0;
    vspec_status st = dev_alloc(&tk->Z, (size_t)tk->sc_max * tk->N * elem, &tot);
    if (st != VSPEC_OK) {
        tk->sc_alloc = 0;
        tk->scratch_bytes -= old_bytes;
        if (tk != plan) plan->scratch_bytes -= old_bytes;
        return st;
    }
    tk->scratch_bytes += tot - old_bytes;
    if (tk != plan) plan->scratch_bytes += tot - old_bytes;
    tk->sc_alloc = tk->sc_max;
    return VSPEC_OK;
}

static vspec_status execute_one(vspec_plan *plan, const int8_t *d_in, int nspectra, float *d_accum,
                                cudaStream_t st);
static vspec_status run_two_kernel(vspec_plan *p, const int8_t *d_in, int nspectra, float *d_accum,
                                   cudaStream_t st, cudaEvent_t before_fold, int band = -1, int nsub = 1);

// The plan a sub-band call of p runs: a fused plan's own two-kernel plan
// (which its long calls run anyway), else p.
static vspec_plan *sb_plan(vspec_plan *p) { return p->fused && p->assist ? p->assist : p; }

// Whether kernel A of plan p can read a band of nsub-band interleaved input
// in place: the dual-pol register-column forms on the plain two-kernel path.
static bool sb_in_place(const vspec_plan *p, int nsub) {
    return nsub > 1 && p->npol == 2 && !p->fused && !p->ring && !p->tc && !p->tc_cols && !p->fir_b && !p->kahan &&
           (std::strcmp(p->formA, "colreg") == 0 || std::strcmp(p->formA, "coldir") == 0);
}

static void make_params(const vspec_plan *p, const int8_t *d_in, int nspectra, vspec::ColParams &ca,
                        vspec::RowParams &cb);

// Whether every band of a sub-band call fits one kernel-A and one kernel-B
// launch per chunk (run_bands): the tiled fold, the slots of nsub bands
// within the plan's partial sums, at least one spectrum of every band in the
// chunk scratch.
static bool bands_fit(const vspec_plan *p, int nsub) {
    if (!sb_in_place(p, nsub) || !p->fold2048 || p->sc_alloc < nsub) return false;
    const int nB = p->blocks_b > 0 ? p->blocks_b : p->num_sms * p->occB;
    const int tilesB = nsub * (p->N2 / p->RB);
    return (nB / tilesB + 2) * nsub <= p->slots_cap;
}

// Every band of a sub-band call in one kernel-A and one kernel-B launch per
// chunk. Kernel A's tile X is column tile X / nsub of band X mod nsub, so
// adjacent tiles (whose CTAs run together) read the same input lines and the
// input comes from HBM once. A spectrum's intermediate holds the bands one
// after another, a virtual spectrum of nsub N points whose nsub N2 rows kernel
// B transforms as usual; the partial sums are slots of that virtual spectrum,
// and one fold per band reads its part.
static vspec_status run_bands(vspec_plan *p, int nsub, const int8_t *d_in, int nspectra, float *d_accum,
                              cudaStream_t st) {
    const int nA = p->blocks_a > 0 ? p->blocks_a : p->num_sms * p->occA;
    const int nB = p->blocks_b > 0 ? p->blocks_b : p->num_sms * p->occB;
    const int cap = std::max(1, std::min(p->sc_max, p->sc_alloc / nsub));  // spectra of all bands in the scratch
    const int nchunks = (nspectra + cap - 1) / cap;
    const int sc_full = (nspectra + nchunks - 1) / nchunks;
    const int tilesB = nsub * (p->N2 / p->RB);
    const long long NV = (long long)nsub * p->N;
    const int slots = (int)(std::min<long long>(nB, (long long)tilesB * sc_full) / tilesB + 2);
    VSPEC_CUDA(cudaMemsetAsync(p->partial, 0, (size_t)slots * NV * sizeof(float4), st));
    vspec::ColParams ca;
    vspec::RowParams cb;
    make_params(p, d_in, nspectra, ca, cb);
    ca.nsub = nsub;
    ca.band = -1;
    ca.zstride = NV;
    ca.tiles = nsub * (p->N1 / p->C);
    cb.N = (int)NV;
    cb.tiles = tilesB;
    cb.slots = slots;
    cb.store = 0;
    for (int s0 = 0; s0 < nspectra; s0 += sc_full) {
        const int sc = std::min(sc_full, nspectra - s0);
        ca.s0 = s0;
        ca.sc = sc;
        void *argsA[] = {&ca};
        int ga = (int)std::min<long long>(nA, (long long)ca.tiles * sc);
        ga = std::max(ca.G, ga / ca.G * ca.G);
        vspec_status r = launch(p, 0, sc * nsub, p->kernelA, dim3(ga), dim3(p->TA), argsA, p->smemA, st);
        if (r != VSPEC_OK) return r;
        cb.s0 = s0;
        cb.sc = sc;
        vspec::TcStatus ts{p->tc_status, g_wait_limit.load()};
        void *argsB[] = {&cb, &ts};
        const int gb = (int)std::min<long long>(nB, (long long)tilesB * sc);
        r = launch(p, 1, sc * nsub, p->kernelB, dim3(gb), dim3(p->TB), argsB, p->smemB, st);
        if (r != VSPEC_OK) return r;
    }
    // one tiled fold per band: its positions are [b N, (b + 1) N) of every slot
    using namespace vspec;
    const int N2 = p->N2, Nv = (int)NV, groups = slots, stride = 1;
    const bool wide = N2 >= 64;
    const void *k = wide ? (const void *)reduce2048_kernel<2, 32, 1> : (const void *)reduce2048_kernel<2, 8, 4>;
    const int *ia = p->invA;
    for (int b = 0; b < nsub; b++) {
        const void *part = reinterpret_cast<const float4 *>(p->partial) + (size_t)b * p->N;
        void *outp = d_accum + (size_t)b * p->N * 4;
        void *argsT[] = {&part, (void *)&groups, (void *)&stride, (void *)&Nv, (void *)&N2, &ia, &outp};
        vspec_status r = launch(p, 2, nspectra, k, dim3(N2 / 16 * 16 * (wide ? 4 : 16)), dim3(wide ? 256 : 512),
                                argsT, 0, st);
        if (r != VSPEC_OK) return r;
    }
    return VSPEC_OK;
}

vspec_status vspec_execute(vspec_plan *plan, const int8_t *d_in, int nspectra, float *d_accum,
                           void *stream) {
    if (!plan || !d_in || !d_accum || nspectra < 0) return VSPEC_ERR_INVALID_ARG;
    if (!aligned16(d_in) || !aligned16(d_accum)) return VSPEC_ERR_ALIGNMENT;
    if (nspectra == 0) return VSPEC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    vspec_plan *p = plan;
    if (p->nsub == 1) return execute_one(p, d_in, nspectra, d_accum, st);
    const int Peff = p->mode == VSPEC_PFB ? p->P : 1;
    const size_t wbytes = (size_t)p->npol * 2;             // one sample of every polarisation
    const size_t outw = (size_t)p->N * (p->npol == 2 ? 4 : 1);
    vspec_plan *t = sb_plan(p);
    if (bands_fit(t, p->nsub)) return run_bands(t, p->nsub, d_in, nspectra, d_accum, st);
    if (sb_in_place(t, p->nsub)) {
        // the register-column kernel A reads each band of the [time][sub][pol]
        // input in place; the bands of a chunk run back to back, so the chunk
        // (about kSbInPlaceBytes of input) comes from HBM once and from L2 after
        const size_t per_spec = (size_t)p->N * p->nsub * wbytes;
        const int chunk = (int)std::max<size_t>(16, kSbInPlaceBytes / per_spec);
        for (int s0 = 0; s0 < nspectra; s0 += chunk) {
            const int cnt = std::min(chunk, nspectra - s0);
            for (int b = 0; b < p->nsub; b++) {
                vspec_status r = run_two_kernel(t, d_in + (size_t)s0 * per_spec, cnt, d_accum + (size_t)b * outw, st,
                                                nullptr, b, p->nsub);
                if (r != VSPEC_OK) return r;
            }
        }
        return VSPEC_OK;
    }
    // other sub-band plans: de-interleave a chunk of spectra, then every sub-band
    const long long slot = (long long)(p->sb_chunk + Peff - 1) * p->N;  // samples per slot
    for (int s0 = 0; s0 < nspectra; s0 += p->sb_chunk) {
        const int cnt = std::min(p->sb_chunk, nspectra - s0);
        const long long M = (long long)(cnt + Peff - 1) * p->N;
        const int8_t *src = d_in + (size_t)s0 * p->N * p->nsub * wbytes;
        const int blocks = (int)((M + 255) / 256);
        const size_t smem = (size_t)256 * (p->nsub + 1) * wbytes;
        if (p->npol == 2)
            vspec::deinterleave_kernel<uint32_t><<<blocks, 256, smem, st>>>(
                reinterpret_cast<const uint32_t *>(src), reinterpret_cast<uint32_t *>(p->sb_scratch),
                p->nsub, M, slot);
        else
            vspec::deinterleave_kernel<uint16_t><<<blocks, 256, smem, st>>>(
                reinterpret_cast<const uint16_t *>(src), reinterpret_cast<uint16_t *>(p->sb_scratch),
                p->nsub, M, slot);
        VSPEC_CUDA(cudaGetLastError());
        for (int b = 0; b < p->nsub; b++) {
            vspec_status r = execute_one(p, p->sb_scratch + (size_t)b * slot * wbytes, cnt,
                                         d_accum + (size_t)b * outw, st);
            if (r != VSPEC_OK) return r;
        }
    }
    return VSPEC_OK;
}

// One-pass fused path: the cluster kernel over all spectra, then the fold of
// its per-cluster partial sums into d_accum.
static vspec_status run_fused(vspec_plan *p, const int8_t *d_in, int nspectra, float *d_accum,
                              cudaStream_t st) {

    if (p->fused_w) {
        vspec::fusedw::Params wp;
        wp.in = d_in;
        wp.coef = p->coef;
        wp.twA = p->twA;
        wp.twB = p->twB;
        wp.twZ = p->twZ;
        wp.partial = reinterpret_cast<float4 *>(p->partial);
        wp.nspectra = nspectra;
        wp.nclusters = p->nclusters;
        void *argsW[] = {&wp};
        vspec_status r = launch(p, 3, nspectra, p->kernelF, dim3(p->cluster * p->nclusters),
                                dim3(vspec::fusedw::kThreads), argsW, p->smemF, st, p->cluster);
        if (r != VSPEC_OK) return r;
        return launch_fold(p, p->nclusters, d_accum, nspectra, st);
    }
    if (p->fused) {
        vspec::fused::Params fp;
        fp.in = d_in;
        fp.coef = p->coef;
        fp.twA = p->twA;
        fp.twB = p->twB;
        fp.twZ = p->twZ;
        fp.partial = reinterpret_cast<float4 *>(p->partial);
        fp.P = p->P;
        fp.nspectra = nspectra;
        fp.nclusters = p->nclusters;
        for (int i = 0; i < vspec::fused::kColPasses; i++) fp.colp[i] = p->passA[i];
        for (int i = 0; i < (int)p->passB.size(); i++) fp.rowp[i] = p->passB[i];
        void *argsF[] = {&fp};
        vspec_status r = launch(p, 3, nspectra, p->kernelF, dim3(p->cluster * p->nclusters),
                                dim3(vspec::fused::kThreads), argsF, p->smemF, st, p->cluster);
        if (r != VSPEC_OK) return r;
        return launch_fold(p, p->nclusters, d_accum, nspectra, st);
    }
    return VSPEC_OK;
}

// Two-kernel path: chunks of column passes (kernel A) and row passes with
// detection (kernel B) through the chunk scratch (in L2 only if a tuned
// chunk is short enough), then the fold of the partial sums into d_accum,
// after `before_fold` if it is given.
// Kernel A's and kernel B's parameters for one call (the per-launch fields,
// chunk start and length, slots and the store flag, are the caller's).
static void make_params(const vspec_plan *p, const int8_t *d_in, int nspectra, vspec::ColParams &ca,
                        vspec::RowParams &cb) {
    ca = vspec::ColParams{};
    ca.in = d_in;
    ca.coef = p->coef;
    ca.twA = p->twA;
    ca.twZ = p->twZ;
    ca.Z = p->Z;
    ca.N = p->N;
    ca.N1 = p->N1;
    ca.N2 = p->N2;
    ca.C = p->C;
    ca.P = p->P;
    ca.lC = ilog2(p->C);
    ca.lN2 = ilog2(p->N2);
    ca.npass = (int)p->passA.size();
    for (int i = 0; i < ca.npass; i++) ca.pass[i] = p->passA[i];
    ca.tiles = p->N1 / p->C;
    ca.G = p->tileG;
    ca.win = p->mode == VSPEC_DIRECT && p->window != VSPEC_WIN_RECT;
    ca.nframes = (long long)nspectra + (p->mode == VSPEC_PFB ? p->P : 1) - 1;
    ca.dftop = p->dftop;
    ca.status = p->tc_status;
    ca.wait_limit = g_wait_limit.load();
    ca.bterms = p->bterms;

    cb = vspec::RowParams{};
    cb.Z = p->Z;
    cb.partial = p->partial;
    cb.partial_comp = p->partial_comp;
    cb.twB = p->twB;
    cb.N = p->N;
    cb.N1 = p->N1;
    cb.N2 = p->N2;
    cb.RB = p->RB;
    cb.lN1 = ilog2(p->N1);
    cb.lRB = ilog2(p->RB);
    cb.npass = (int)p->passB.size();
    for (int i = 0; i < cb.npass; i++) cb.pass[i] = p->passB[i];
    cb.tiles = p->N2 / p->RB;
    cb.in = d_in;
    cb.coef = p->coef;
    cb.P = p->P;
    cb.nframes = ca.nframes;
}

static vspec_status run_two_kernel(vspec_plan *p, const int8_t *d_in, int nspectra, float *d_accum,
                                   cudaStream_t st, cudaEvent_t before_fold, int band, int nsub) {
    const size_t accel = p->npol == 2 ? sizeof(float4) : sizeof(float);
    // one full wave of CTAs per launch unless tuned; the work is split evenly
    // over them (block_span), so every SM stays busy to the end of a launch
    const int nA = p->blocks_a > 0 ? p->blocks_a : p->num_sms * p->occA;
    const int nB = p->blocks_b > 0 ? p->blocks_b : p->num_sms * p->occB;
    // equal chunks of at most sc_max spectra (no short ragged last chunk)
    const int nchunks = (nspectra + p->sc_max - 1) / p->sc_max;
    const int sc_full = (nspectra + nchunks - 1) / nchunks;
    // slots of the largest kernel-B launch (no more CTAs than items)
    const int tilesB = p->N2 / p->RB;
    int slots = slots_for(p, (int)std::min<long long>(nB, (long long)tilesB * sc_full));
    // a one-row transform in one launch: block k is the only writer of slot k
    // and stores it, so nothing needs zeroing and the fold reads those slots
    const bool store = p->fir_b && !p->kahan && !p->tc && nchunks == 1;
    if (store) slots = (int)std::min<long long>(nB, (long long)tilesB * sc_full);
    if (!store) VSPEC_CUDA(cudaMemsetAsync(p->partial, 0, (size_t)slots * p->N * accel, st));
    if (p->kahan) VSPEC_CUDA(cudaMemsetAsync(p->partial_comp, 0, (size_t)slots * p->N * accel, st));

    vspec::ColParams ca;
    vspec::RowParams cb;
    make_params(p, d_in, nspectra, ca, cb);
    cb.slots = slots;
    cb.store = store;
    if (band >= 0) {  // kernel A reads band `band` of the nsub-band [time][sub][pol] input in place
        ca.nsub = nsub;
        ca.band = band;
    }

    for (int s0 = 0; s0 < nspectra; s0 += sc_full) {
        const int sc = std::min(sc_full, nspectra - s0);
        if (!p->fir_b) {
            ca.s0 = s0;
            ca.sc = sc;
            void *argsA[] = {&ca};
            // no more CTAs than items, and a whole number of tile groups
            int ga = (int)std::min<long long>(nA, (long long)ca.tiles * sc);
            ga = std::max(ca.G, ga / ca.G * ca.G);
            vspec_status r = launch(p, 0, sc, p->kernelA, dim3(ga), dim3(p->TA), argsA, p->smemA, st);
            if (r != VSPEC_OK) return r;
        }
        vspec_status r;
        cb.s0 = s0;
        cb.sc = sc;
        vspec::TcStatus ts{p->tc_status, g_wait_limit.load()};
        void *argsB[] = {&cb, &ts};
        const int gb = (int)std::min<long long>(nB, (long long)cb.tiles * sc);
        r = launch(p, 1, sc, p->kernelB, dim3(gb), dim3(p->TB), argsB, p->smemB, st);
        if (r != VSPEC_OK) return r;
    }
    if (before_fold) VSPEC_CUDA(cudaStreamWaitEvent(st, before_fold, 0));
    return launch_fold(p, slots, d_accum, nspectra, st);
}

// The persistent ring form: one cooperative launch per kRingSlotsPerLaunch
// slots (each with its done counters zeroed first), then the fold of the
// partial-sum sets in set order.
static vspec_status run_ring(vspec_plan *p, const int8_t *d_in, int nspectra, float *d_accum, cudaStream_t st) {
    if (p->ringS == 0 || !p->Z || !p->partial) {
        g_last_error = "the ring plan has no ring (a reshape failed)";
        return VSPEC_ERR_OOM;
    }
    const int S = p->ringS, V = p->ringV;
    const long long nslot_all = ((long long)nspectra + S - 1) / S;
    // set cycle: about 32 slot sums per set, at least 2 (B(c) then waits for B(c - K) only)
    const int K = (int)std::min<long long>(p->ring_sets / V, std::max<long long>(2, (nslot_all + 31) / 32));
    vspec::RingParams q{};
    make_params(p, d_in, nspectra, q.a, q.b);
    q.ring = p->Z;
    q.sets = p->partial;
    q.status = p->tc_status;
    q.wait_limit = g_wait_limit.load();
    q.S = S;
    q.R = p->ringR;
    q.L = p->ringL;
    q.V = V;
    q.K = K;
    q.tilesA = p->N1 / p->C;
    q.tilesB = p->N2;
    q.discard = p->ring_discard;
    for (long long c0 = 0; c0 < nslot_all; c0 += kRingSlotsPerLaunch) {
        q.nslot = (int)std::min<long long>(kRingSlotsPerLaunch, nslot_all - c0);
        q.c0 = (int)c0;
        q.s0 = c0 * S;
        q.nspectra = (int)std::min<long long>((long long)nspectra - c0 * S, (long long)q.nslot * S);
        q.ctl = p->ring_ctl;
        VSPEC_CUDA(cudaMemsetAsync(p->ring_ctl, 0, sizeof(int) * (2 + 2 * (size_t)q.nslot), st));
        if (p->ring_stall >= 0 && p->ring_stall < q.nslot) {
            // failure injection: one more A ticket than slot ring_stall has, so its B tickets' wait gives up
            VSPEC_CUDA(cudaMemsetAsync(p->ring_ctl + 2 + p->ring_stall, 0xff, sizeof(int), st));  // -1
            p->ring_stall = -1;
        }
        void *args[] = {&q};
        vspec_status r = launch(p, 3, q.nspectra, p->kernelRing, dim3(p->ring_grid), dim3(512), args, p->smemRing,
                                st, -1);
        if (r != VSPEC_OK) return r;
    }
    return launch_fold(p, (int)std::min<long long>(K, nslot_all) * V, d_accum, nspectra, st);
}

}  // extern "C"

// ------------------------------------------------ persistent multi-bank --
// (C++ linkage: declared in vspec_internal.h for vspec_batch.cu)
// The plan whose forms a bank of the persistent launch runs: a fused plan's
// own two-kernel plan (which its long calls run anyway), else the plan.
static vspec_plan *bp_plan(vspec_plan *p) { return p->fused && p->assist ? p->assist : p; }

// Ticket body of a plan in the persistent multi-bank launch, -1 if none.
static int bp_form(const vspec_plan *p0, const char **why) {
    const vspec_plan *p = bp_plan(const_cast<vspec_plan *>(p0));
    const char *w = nullptr;
    int f = -1;
    if (p->npol != 2 || p->fused || p->kahan || p->tc || p->tc_cols || p->ring || p0->nsub != 1)
        w = "needs a dual-pol two-kernel FP32 plan (VSPEC_PLAN_TWO_KERNEL) without sub-bands";
    else if (p->fir_b && p->N == 2048 && std::strcmp(p->formB, "row2048") == 0)
        f = vspec::kBpRow2048Fir;
    else if (p->fir_b && p->N <= 1024 && p->P <= 8 && p->RB == 1)
        f = vspec::kBpRowFir;
    else if (!p->fir_b && std::strcmp(p->formB, "row2048") == 0 && std::strcmp(p->formA, "colreg") == 0)
        f = vspec::kBpColreg;
    else if (!p->fir_b && std::strcmp(p->formB, "row2048") == 0 && std::strcmp(p->formA, "coldir") == 0)
        f = vspec::kBpColdir;
    else
        w = "needs the register-column kernel A with 2048-point rows (PFB of 5..8 taps up to 2^18 channels, "
            "direct mode up to 2^19) or a one-row transform (up to 1024 channels with at most 8 taps, or 2048)";
    if (why) *why = w;
    return f;
}

void vspec_set_last_error(const char *what) { g_last_error = what ? what : ""; }

vspec_status vspec_bp_supported(const vspec_plan *p, const char **why) {
    if (!p) return VSPEC_ERR_INVALID_ARG;
    return bp_form(p, why) >= 0 ? VSPEC_OK : VSPEC_ERR_UNSUPPORTED;
}

vspec_status vspec_bp_execute(vspec_plan *const *plans, int n, const int8_t *const *d_in, const int *nspectra,
                              float *const *d_accum, int *ctl, int *status, int stall_bank, cudaStream_t st) {
    using namespace vspec;
    if (!plans || !d_in || !nspectra || !d_accum || !ctl || n < 1) return VSPEC_ERR_INVALID_ARG;
    if (n > kBpMaxBanks) {
        g_last_error = "the persistent launch holds at most 16 banks";
        return VSPEC_ERR_UNSUPPORTED;
    }
    static BpParams q;  // about 10 KB of kernel parameters (callers are serialised per batch)
    static std::mutex q_mutex;
    std::lock_guard<std::mutex> lock(q_mutex);
    q = BpParams{};
    size_t smem = 0;
    q.nbanks = n;
    // banks in the caller's order (decreasing size measured 4% slower on the
    // eight-bank workload)
    int order[kBpMaxBanks];
    for (int i = 0; i < n; i++) order[i] = i;
    for (int j = 0; j < n; j++) {
        const int i = order[j];
        vspec_plan *p = plans[i] ? bp_plan(plans[i]) : nullptr;
        const char *why = nullptr;
        const int form = p ? bp_form(p, &why) : -1;
        if (form < 0) {
            g_last_error = why ? why : "missing plan";
            return p ? VSPEC_ERR_UNSUPPORTED : VSPEC_ERR_INVALID_ARG;
        }
        const int ns = nspectra[i];
        if (ns < 0 || !d_in[i] || !d_accum[i]) return VSPEC_ERR_INVALID_ARG;
        if (!aligned16(d_in[i]) || !aligned16(d_accum[i])) return VSPEC_ERR_ALIGNMENT;
        const bool rowonly = form == kBpRowFir || form == kBpRow2048Fir;
        if (!rowonly && ns > p->sc_alloc) {
            g_last_error = "a bank's call is longer than its plan's chunk scratch (tune chunk_spectra to the call)";
            return VSPEC_ERR_UNSUPPORTED;
        }
        BpBank &b = q.banks[j];
        make_params(p, d_in[i], ns, b.a, b.b);
        b.a.s0 = 0;
        b.a.sc = ns;
        b.b.s0 = 0;
        b.b.sc = ns;
        b.Z = p->Z;
        b.sets = reinterpret_cast<float4 *>(p->partial);
        b.acc = reinterpret_cast<float4 *>(d_accum[i]);
        b.invA = p->invA;
        b.invB = p->invB;
        b.form = form;
        b.N2 = p->N2;
        b.nspectra = ns;
        // tickets of about 40 us of work: 128 spectra of a 512-point PFB tile,
        // 32 of a 2048-point direct tile, 32 of a row (16 per group, one
        // register run)
        b.TA = form == kBpColreg ? 128 : 32;
        b.TB = 32;
        if ((ns + b.TB - 1) / b.TB > p->slots_cap) {
            g_last_error = "a bank's call needs more partial-sum sets than its plan holds";
            return VSPEC_ERR_UNSUPPORTED;
        }
        b.tilesA = rowonly ? 0 : p->N1 / p->C;
        b.tilesB = rowonly ? 1 : p->N2;
        b.nA = ns > 0 ? b.tilesA * ((ns + b.TA - 1) / b.TA) : 0;
        b.nB = ns > 0 ? b.tilesB * ((ns + b.TB - 1) / b.TB) : 0;
        b.nF = ns > 0 ? (p->N + kBpFoldChannels - 1) / kBpFoldChannels : 0;
        if (!rowonly) smem = std::max(smem, vspec_bp_smem_a(form, p->N2));
        smem = std::max(smem, vspec_bp_smem_b(form, p->N1, p->P));
        q.offA[j + 1] = q.offA[j] + b.nA;
        q.offB[j + 1] = q.offB[j] + b.nB;
        q.offF[j + 1] = q.offF[j] + b.nF;
    }
    q.ctl = ctl;
    q.status = status;
    q.wait_limit = g_wait_limit.load();
    vspec_plan *p0 = bp_plan(plans[0]);
    const void *fn = vspec_bp_kernel();
    static std::once_flag raised;
    static cudaError_t raise_err = cudaSuccess;
    std::call_once(raised, [&] { raise_err = raise_smem_cap(fn, 232448 - 64); });
    VSPEC_CUDA(raise_err);
    int occ = 0;
    VSPEC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 512, smem));
    if (occ < 1) {
        g_last_error = "the multi-bank kernel does not fit on an SM";
        return VSPEC_ERR_UNSUPPORTED;
    }
    VSPEC_CUDA(cudaMemsetAsync(ctl, 0, sizeof(int) * (2 + 2 * (size_t)n), st));
    for (int j = 0; j < n; j++)  // the injected stall, at the bank's place in the kernel's order
        if (order[j] == stall_bank) VSPEC_CUDA(cudaMemsetAsync(ctl + 2 + 2 * j, 0xff, sizeof(int), st));
    int spectra = 0;
    for (int i = 0; i < n; i++) spectra += nspectra[i];
    void *args[] = {&q};
    return launch(p0, 3, spectra, fn, dim3(p0->num_sms * occ), dim3(512), args, smem, st, -1);
}

extern "C" {

static vspec_status execute_one(vspec_plan *p, const int8_t *d_in, int nspectra, float *d_accum,
                                cudaStream_t st) {
    if (p->ring) return run_ring(p, d_in, nspectra, d_accum, st);
    if (!p->fused) return run_two_kernel(p, d_in, nspectra, d_accum, st, nullptr);
    if (p->assist && nspectra >= p->two_kernel_from)
        return run_two_kernel(p->assist, d_in, nspectra, d_accum, st, nullptr);
    const int sa = p->assist ? (int)((long long)nspectra * p->assist_permille / 1000) : 0;
    if (sa < kAssistMinSpectra) return run_fused(p, d_in, nspectra, d_accum, st);
    // fused kernel on `st` over the first spectra, the assist plan on its own
    // stream over the rest; the two folds into d_accum are ordered
    const int sf = nspectra - sa;
    VSPEC_CUDA(cudaEventRecord(p->ev_fork, st));
    VSPEC_CUDA(cudaStreamWaitEvent(p->assist_st, p->ev_fork, 0));
    vspec_status r = run_fused(p, d_in, sf, d_accum, st);
    if (r != VSPEC_OK) return r;
    VSPEC_CUDA(cudaEventRecord(p->ev_main, st));
    r = run_two_kernel(p->assist, d_in + (size_t)sf * p->N * p->npol * 2, sa, d_accum, p->assist_st,
                       p->ev_main);
    if (r != VSPEC_OK) return r;
    VSPEC_CUDA(cudaEventRecord(p->ev_assist, p->assist_st));
    VSPEC_CUDA(cudaStreamWaitEvent(st, p->ev_assist, 0));
    return VSPEC_OK;
}

vspec_status vspec_plan_set_profiling(vspec_plan *plan, int enable) {
    if (!plan) return VSPEC_ERR_INVALID_ARG;
    for (auto &r : plan->recs) cudaEventSynchronize(r.stop);
    release_records(plan);
    plan->profiling = enable != 0;
    return VSPEC_OK;
}

vspec_status vspec_plan_kernel_stats(vspec_plan *plan, int kind, int reset, const char **name,
                                     long long *launches, long long *spectra, double *total_ms) {
    if (!plan || kind < 0 || kind >= kNumKinds) return VSPEC_ERR_INVALID_ARG;
    long long n = 0, sp = 0;
    double ms = 0.0;
    for (auto &r : plan->recs) {
        if (r.kind != kind) continue;
        VSPEC_CUDA(cudaEventSynchronize(r.stop));
        float t = 0.f;
        VSPEC_CUDA(cudaEventElapsedTime(&t, r.start, r.stop));
        ms += t;
        n++;
        sp += r.spectra;
    }
    if (name) *name = kKindNames[kind];
    if (launches) *launches = n;
    if (spectra) *spectra = sp;
    if (total_ms) *total_ms = ms;
    if (reset) {
        for (auto &r : plan->recs) cudaEventSynchronize(r.stop);
        release_records(plan);
    }
    return VSPEC_OK;
}

// Spectra per chunk of the host-input pipeline: about host_chunk_bytes of
// input per staging buffer (at least 16 spectra), so copies and compute
// overlap; the pipeline exposes one chunk's copy at the start and one
// chunk's compute at the end. Automatic (host_chunk_bytes == 0): a sixteenth
// of the first call's input, within 32 .. 256 MiB, so that the exposed ends
// stay small while each chunk's fixed costs (launches, the P - 1 frames read
// twice) are spread over more spectra.
static int host_chunk_spectra(const vspec_plan *p, int nspectra) {
    const size_t per = (size_t)p->N * p->nsub * p->npol * 2;
    size_t bytes = p->host_chunk_bytes;
    if (bytes == 0)
        bytes = std::min<size_t>(256u << 20, std::max<size_t>(32u << 20, (size_t)nspectra * per / 16));
    return (int)std::max<size_t>(16, bytes / per);
}

vspec_status vspec_execute_host(vspec_plan *plan, const int8_t *h_in, int nspectra, float *h_out,
                                void *stream) {
    if (!plan || !h_in || !h_out || nspectra < 0) return VSPEC_ERR_INVALID_ARG;
    vspec_plan *p = plan;
    cudaStream_t st = (cudaStream_t)stream;
    const int Peff = p->mode == VSPEC_PFB ? p->P : 1;
    const size_t frame = (size_t)p->N * p->nsub * p->npol * 2;
    const size_t out_bytes = (size_t)p->nsub * p->N * (p->npol == 2 ? 4 : 1) * sizeof(float);
    if (!p->host_ready) {
        p->stage_spectra = host_chunk_spectra(p, nspectra);
        const size_t sbytes = (size_t)(p->stage_spectra + Peff - 1) * frame;
        size_t tot = 0;
        vspec_status r;
        for (int b = 0; b < 2; b++)
            if ((r = dev_alloc((void **)&p->stage[b], sbytes, &tot))) return r;
        if ((r = dev_alloc((void **)&p->hacc, out_bytes, &tot))) return r;
        VSPEC_CUDA(cudaStreamCreateWithFlags(&p->copy_st, cudaStreamNonBlocking));
        VSPEC_CUDA(cudaStreamCreateWithFlags(&p->comp_st, cudaStreamNonBlocking));
        VSPEC_CUDA(cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming));
        VSPEC_CUDA(cudaEventCreateWithFlags(&p->ev_done, cudaEventDisableTiming));
        for (int b = 0; b < 2; b++) {
            VSPEC_CUDA(cudaEventCreateWithFlags(&p->ev_copied[b], cudaEventDisableTiming));
            VSPEC_CUDA(cudaEventCreateWithFlags(&p->ev_used[b], cudaEventDisableTiming));
        }
        p->scratch_bytes += tot;
        p->host_bytes = tot;
        p->host_ready = true;
    }
    // both internal streams start after the work already queued on `stream`
    VSPEC_CUDA(cudaEventRecord(p->ev_start, st));
    VSPEC_CUDA(cudaStreamWaitEvent(p->copy_st, p->ev_start, 0));
    VSPEC_CUDA(cudaStreamWaitEvent(p->comp_st, p->ev_start, 0));
    VSPEC_CUDA(cudaMemsetAsync(p->hacc, 0, out_bytes, p->comp_st));

    // mapped input: the kernels read the pinned host buffer through its
    // device address
    const int8_t *mapped = nullptr;
    if (p->host_mode != VSPEC_HOST_STAGED) {
        cudaPointerAttributes attr{};
        if (cudaPointerGetAttributes(&attr, h_in) == cudaSuccess && attr.type == cudaMemoryTypeHost &&
            attr.devicePointer != nullptr)
            mapped = static_cast<const int8_t *>(attr.devicePointer);
        else
            cudaGetLastError();  // clear a lookup failure on unregistered memory
        if (!mapped && p->host_mode == VSPEC_HOST_MAPPED) {
            g_last_error = "vspec_execute_host: h_in is not pinned host memory the device can address";
            return VSPEC_ERR_INVALID_ARG;
        }
    }
    if (mapped) {
        vspec_status r = vspec_execute(p, mapped, nspectra, p->hacc, (void *)p->comp_st);
        if (r != VSPEC_OK) return r;
        VSPEC_CUDA(cudaMemcpyAsync(h_out, p->hacc, out_bytes, cudaMemcpyDeviceToHost, p->comp_st));
        VSPEC_CUDA(cudaEventRecord(p->ev_done, p->comp_st));
        VSPEC_CUDA(cudaStreamWaitEvent(st, p->ev_done, 0));
        return VSPEC_OK;
    }
    const int chunk = p->stage_spectra;
    int k = 0;
    for (int s0 = 0; s0 < nspectra; s0 += chunk, k++) {
        const int cnt = std::min(chunk, nspectra - s0);
        const int b = k & 1;
        // the buffer is free once the compute that read it two chunks ago is done
        if (k >= 2) VSPEC_CUDA(cudaStreamWaitEvent(p->copy_st, p->ev_used[b], 0));
        VSPEC_CUDA(cudaMemcpyAsync(p->stage[b], h_in + (size_t)s0 * frame, (size_t)(cnt + Peff - 1) * frame,
                                   cudaMemcpyHostToDevice, p->copy_st));
        VSPEC_CUDA(cudaEventRecord(p->ev_copied[b], p->copy_st));
        VSPEC_CUDA(cudaStreamWaitEvent(p->comp_st, p->ev_copied[b], 0));
        vspec_status r = vspec_execute(p, p->stage[b], cnt, p->hacc, (void *)p->comp_st);
        if (r != VSPEC_OK) return r;
        VSPEC_CUDA(cudaEventRecord(p->ev_used[b], p->comp_st));
    }
    VSPEC_CUDA(cudaMemcpyAsync(h_out, p->hacc, out_bytes, cudaMemcpyDeviceToHost, p->comp_st));
    VSPEC_CUDA(cudaEventRecord(p->ev_done, p->comp_st));
    VSPEC_CUDA(cudaStreamWaitEvent(st, p->ev_done, 0));
    return VSPEC_OK;
}

vspec_status vspec_plan_set_host_mode(vspec_plan *plan, int mode, size_t chunk_bytes) {
    if (!plan || mode < VSPEC_HOST_AUTO || mode > VSPEC_HOST_MAPPED) return VSPEC_ERR_INVALID_ARG;
    if (chunk_bytes != 0 && (chunk_bytes < (1u << 20) || chunk_bytes > (1ull << 32))) return VSPEC_ERR_INVALID_ARG;
    const size_t bytes = chunk_bytes;  // 0: automatic
    if (plan->host_ready && bytes != plan->host_chunk_bytes) {  // staging buffers are sized by the chunk
        VSPEC_CUDA(cudaDeviceSynchronize());
        release_host_pipeline(plan);
    }
    plan->host_mode = mode;
    plan->host_chunk_bytes = bytes;
    return VSPEC_OK;
}

vspec_status vspec_plan_check(vspec_plan *plan) {
    if (!plan) return VSPEC_ERR_INVALID_ARG;
    if (!plan->tc_status) return VSPEC_OK;
    int h = 0;
    VSPEC_CUDA(cudaMemcpy(&h, plan->tc_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (!h) return VSPEC_OK;
    VSPEC_CUDA(cudaMemset(plan->tc_status, 0, sizeof(int)));
    g_last_error = "a bounded wait for the tensor cores expired";
    return VSPEC_ERR_DEVICE_TIMEOUT;
}

vspec_status vspec_debug_flags(unsigned *flags, int clear) {
#ifdef VSPEC_DEBUG
    if (!flags) return VSPEC_ERR_INVALID_ARG;
    VSPEC_CUDA(cudaDeviceSynchronize());
    VSPEC_CUDA(cudaMemcpyFromSymbol(flags, vspec::g_debug_flags, sizeof(unsigned)));
    if (clear) {
        const unsigned zero = 0;
        VSPEC_CUDA(cudaMemcpyToSymbol(vspec::g_debug_flags, &zero, sizeof(unsigned)));
    }
    unsigned ring_flags = 0, bp_flags = 0;  // the ring and multi-bank kernels' own words
    VSPEC_CUDA(vspec_ring_debug_flags(&ring_flags, clear != 0));
    VSPEC_CUDA(vspec_bp_debug_flags(&bp_flags, clear != 0));
    *flags |= ring_flags | bp_flags;
    return VSPEC_OK;
#else
    (void)flags;
    (void)clear;
    g_last_error = "bounds checks are compiled only into the debug build (VSPEC_DEBUG)";
    return VSPEC_ERR_UNSUPPORTED;
#endif
}

vspec_status vspec_set_wait_limit(long long polls) {
    if (polls > (long long)UINT32_MAX) return VSPEC_ERR_INVALID_ARG;
    g_wait_limit.store(polls < 0 ? vspec::tc::kSpinLimit : (uint32_t)polls);
    return VSPEC_OK;
}

vspec_status vspec_plan_inject_timeout(vspec_plan *plan) {
    if (!plan) return VSPEC_ERR_INVALID_ARG;
    if (!plan->tc_status) {
        g_last_error = "this plan has no bounded device-side wait";
        return VSPEC_ERR_UNSUPPORTED;
    }
    const int one = 1;
    VSPEC_CUDA(cudaMemcpy(plan->tc_status, &one, sizeof(int), cudaMemcpyHostToDevice));
    return VSPEC_OK;
}

vspec_status vspec_plan_inject_stall(vspec_plan *plan, int slot) {
    if (!plan || slot < 0) return VSPEC_ERR_INVALID_ARG;
    if (!plan->ring) {
        g_last_error = "only ring plans wait on other CTAs' work";
        return VSPEC_ERR_UNSUPPORTED;
    }
    plan->ring_stall = slot;
    return VSPEC_OK;
}

vspec_status vspec_tc_dft16(const float *d_x, float *d_y, int batch, int terms, void *stream) {
    if (!d_x || !d_y || batch < 0 || (terms != 1 && terms != 3)) return VSPEC_ERR_INVALID_ARG;
    if (!aligned16(d_x) || !aligned16(d_y)) return VSPEC_ERR_ALIGNMENT;
    if (batch == 0) return VSPEC_OK;
    static int *d_status = nullptr;  // one int per process for the bounded-wait flag
    if (!d_status) VSPEC_CUDA(cudaMalloc(&d_status, sizeof(int)));
    cudaStream_t st = (cudaStream_t)stream;
    VSPEC_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), st));
    vspec::tc::dft16_kernel<<<(batch + 127) / 128, 128, 0, st>>>(
        reinterpret_cast<const float2 *>(d_x), reinterpret_cast<float2 *>(d_y), batch, terms, d_status,
        g_wait_limit.load());
    VSPEC_CUDA(cudaGetLastError());
    int h = 0;
    VSPEC_CUDA(cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    VSPEC_CUDA(cudaStreamSynchronize(st));
    return h ? VSPEC_ERR_DEVICE_TIMEOUT : VSPEC_OK;
}

vspec_status vspec_dump(vspec_plan *plan, float *d_accum, float *h_out, void *stream) {
    if (!plan || !d_accum) return VSPEC_ERR_INVALID_ARG;
    if (!aligned16(d_accum)) return VSPEC_ERR_ALIGNMENT;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)plan->nsub * plan->N * (plan->npol == 2 ? 4 : 1) * sizeof(float);
    if (h_out) VSPEC_CUDA(cudaMemcpyAsync(h_out, d_accum, bytes, cudaMemcpyDeviceToHost, st));
    VSPEC_CUDA(cudaMemsetAsync(d_accum, 0, bytes, st));
    if (plan->out_comp) VSPEC_CUDA(cudaMemsetAsync(plan->out_comp, 0, bytes / plan->nsub, st));
    return VSPEC_OK;
}

}  // extern "C"

// ===================================================== allocation-free path ===
//
// vspec_execute_noalloc channelizes like vspec_execute, with the generic
// two-kernel form of the path (general kernel A, general row kernel B, plain
// fold), and keeps its coefficients, twiddle tables, digit-reversal maps,
// chunk scratch and partial sums in one fixed device array declared below
// instead of memory from cudaMalloc. It exists for callers that cannot allocate device memory:
// a host application that owns every byte of device memory through its own
// pool, or a real-time capture loop where a cudaMalloc (which can synchronise
// the whole device) would stall the data path and drop samples. The paper
// has no counterpart.

namespace {

constexpr int kNoAllocMaxChan = 32768;  // largest nchan the fixed array holds
constexpr int kNoAllocChunk = 16;       // spectra per scratch chunk
constexpr int kNoAllocGroups = 16;      // kernel-B partial-sum slots
constexpr int kMaxDevices = 64;

// byte offsets inside the array (every region 256-byte aligned)
constexpr size_t kNaCoef = 0;                                            // 16 * N floats
constexpr size_t kNaTwA = kNaCoef + 16ull * kNoAllocMaxChan * 4;         // < N float2
constexpr size_t kNaTwB = kNaTwA + (size_t)kNoAllocMaxChan * 8;          // < N float2
constexpr size_t kNaTwZ = kNaTwB + (size_t)kNoAllocMaxChan * 8;          // N float2
constexpr size_t kNaInts = kNaTwZ + (size_t)kNoAllocMaxChan * 8;         // kA, invA, invB
constexpr size_t kNaZ = kNaInts + 3ull * kNoAllocMaxChan * 4;            // chunk scratch
constexpr size_t kNaPartial = kNaZ + (size_t)kNoAllocChunk * kNoAllocMaxChan * 16;
constexpr size_t kNoAllocBytes = kNaPartial + (size_t)kNoAllocGroups * kNoAllocMaxChan * 16;

// The fixed scratch: 20 MiB, held by every GPU that loads this library until
// the process exits. Host code must not pass this name to a kernel: on the
// host it is only a stand-in; its device address comes from
// cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocCfg {
    int N, P, npol, mode, window;
    int N1, N2, C, PT, PPT, TA, RB, TB, sc_max, occA;
    int blocks_a, blocks_b, slots;  // CTAs per launch; partial-sum slots
    int nA, nB;
    Pass passA[vspec::kMaxPasses], passB[vspec::kMaxPasses];
    const void *kA, *kB, *kR;
    size_t smemA, smemB;
};

struct NoAllocDevice {
    bool ready = false;
    unsigned char *base = nullptr;  // device address of g_noalloc_scratch
    int num_sms = 0;
    bool tables_valid = false;
    int key[5] = {0, 0, 0, 0, 0};   // (N, P, npol, mode, window) of the tables
};

std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_dev[kMaxDevices];

// Digit-reversal maps of both DFT factors, computed on the device:
// kA[pos] = k2 held at row position pos, invA[k2] = pos, invB[k1] = posB.
__global__ void noalloc_digrev_kernel(int *kA, int *invA, int *invB, int N2, int N1,
                                      NoAllocCfg cfg) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < N2) {
        int rem = e, lb = N2, k = 0, scale = 1;
        for (int i = 0; i < cfg.nA; i++) {
            const int m = lb / cfg.passA[i].r, q = rem / m;
            rem -= q * m;
            k += q * scale;
            scale *= cfg.passA[i].r;
            lb = m;
        }
        kA[e] = k;
        invA[k] = e;
    }
    if (e < N1) {
        int rem = e, lb = N1, k = 0, scale = 1;
        for (int i = 0; i < cfg.nB; i++) {
            const int m = lb / cfg.passB[i].r, q = rem / m;
            rem -= q * m;
            k += q * scale;
            scale *= cfg.passB[i].r;
            lb = m;
        }
        invB[k] = e;
    }
}

// Sizes of the generic two-kernel form for nchan <= 32768: the four-step
// split of build_plan (rows of at most 2048 points), with narrower column
// tiles (16 or 32 byte rows, 256-point tiles) and short chunks, so that the
// scratch fits the fixed array. build_plan's faster kernel forms (register
// columns, the 2048-point row kernel, the tiled fold, the cluster kernel) are
// not used here, so results agree with vspec_execute within the FP32
// tolerance, not bit for bit.
vspec_status noalloc_configure(NoAllocCfg *c, int num_sms) {
    const int N = c->N;
    const bool pfb = c->mode == VSPEC_PFB;
    const int PT = c->P <= 1 ? 1 : c->P <= 2 ? 2 : c->P <= 4 ? 4 : c->P <= 8 ? 8 : 16;
    const int cmin = c->npol == 2 ? 16 : 32;
    int n2max = !pfb ? 4096 / cmin : PT <= 8 ? 1024 / cmin : 512 / cmin;
    int N2 = 1;
    while (N / N2 > kRowElems && N2 < n2max) N2 *= 2;
    const int N1 = N / N2;
    int C = std::min(std::max(cmin, 256 / N2), N1);
    const int pts = N2 * C;
    c->TA = std::min(512, pts);
    c->PPT = pts / c->TA;
    c->N1 = N1;
    c->N2 = N2;
    c->C = C;
    c->PT = PT;
    c->kA = c->npol == 2 ? pick_kernel_a<2>(PT, c->PPT) : pick_kernel_a<1>(PT, c->PPT);
    if (!c->kA) {
        g_last_error = "no kernel instance for this tap count and size";
        return VSPEC_ERR_UNSUPPORTED;
    }
    c->kB = c->npol == 2 ? (const void *)vspec::rowfft_detect_kernel<2> : (const void *)vspec::rowfft_detect_kernel<1>;
    c->kR = c->npol == 2 ? (const void *)vspec::reduce_kernel<2> : (const void *)vspec::reduce_kernel<1>;
    const int capA = vspec::col_radix_cap(c->npol, PT, c->PPT);
    const int e = ilog2(N), e2 = ilog2(N2);
    // pass lists as in radix_list / make_passes, in fixed arrays (no heap)
    auto fill = [](Pass *ps, int L, int ebits, int maxbits) {
        int np = ebits == 0 ? 0 : (ebits + maxbits - 1) / maxbits;
        int lb = L, off = 0;
        for (int i = 0; i < np; i++) {
            const int r = 1 << (ebits / np + (i < ebits % np ? 1 : 0));
            ps[i].r = r;
            ps[i].lb = lb;
            ps[i].m = lb / r;
            ps[i].off = off;
            ps[i].lr = ilog2(r);
            ps[i].lm = ilog2(lb / r);
            off += ps[i].m * (r - 1);
            lb /= r;
        }
        return np;
    };
    c->nA = fill(c->passA, N2, e2, capA == 16 ? 4 : capA == 8 ? 3 : 2);
    c->nB = fill(c->passB, N1, e - e2, 4);
    c->RB = std::max(1, std::min(N2, kRowElems / N1));
    int maxb = 1;
    for (int i = 0; i < c->nB; i++) maxb = std::max(maxb, c->RB * (N1 / c->passB[i].r));
    c->TB = std::min(256, std::max(32, maxb));
    const size_t elem = c->npol == 2 ? sizeof(float4) : sizeof(float2);
    const size_t accel = c->npol == 2 ? sizeof(float4) : sizeof(float);
    c->smemA = (size_t)PT * N2 * C * elem + (size_t)N2 * C * sizeof(float2) +
               2 * (size_t)PT * N2 * C * c->npol * 2;  // + twiddle tile, raw frames
    c->smemB = (size_t)c->RB * (N1 + (N1 >> 4)) * elem + (size_t)c->RB * N1 * accel;
    VSPEC_CUDA(raise_smem_cap(c->kA, c->smemA));
    VSPEC_CUDA(raise_smem_cap(c->kB, c->smemB));
    int occB = 1;
    VSPEC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->occA, c->kA, c->TA, c->smemA));
    VSPEC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occB, c->kB, c->TB, c->smemB));
    c->sc_max = (int)std::min<size_t>(kNoAllocChunk, (size_t)kNoAllocChunk * kNoAllocMaxChan / N);
    // one wave of CTAs per launch, as many kernel-B CTAs as the slots allow
    const int tilesB = N2 / c->RB;
    c->blocks_a = num_sms * std::max(1, c->occA);
    c->blocks_b = std::min(num_sms * std::max(1, occB), (kNoAllocGroups - 2) * tilesB);
    c->slots = c->blocks_b / tilesB + 2;
    return VSPEC_OK;
}

}  // namespace

extern "C" vspec_status vspec_execute_noalloc(const int8_t *d_in, int nchan, int ntaps, int npol,
                                              vspec_mode mode, vspec_window window, int nspectra,
                                              float *d_accum, void *stream) {
    if (!d_in || !d_accum || nspectra < 0) return VSPEC_ERR_INVALID_ARG;
    if (!is_pow2(nchan) || nchan < 16 || nchan > (1 << 20)) return VSPEC_ERR_INVALID_ARG;
    if (npol != 1 && npol != 2) return VSPEC_ERR_INVALID_ARG;
    if (mode != VSPEC_PFB && mode != VSPEC_DIRECT) return VSPEC_ERR_INVALID_ARG;
    if (window != VSPEC_WIN_RECT && window != VSPEC_WIN_HANN && window != VSPEC_WIN_HAMMING)
        return VSPEC_ERR_INVALID_ARG;
    if (mode == VSPEC_PFB && (ntaps < 1 || ntaps > 16)) return VSPEC_ERR_INVALID_ARG;
    if (mode == VSPEC_DIRECT && (ntaps < 0 || ntaps > 1)) return VSPEC_ERR_INVALID_ARG;
    if (nchan > kNoAllocMaxChan) {
        g_last_error = "vspec_execute_noalloc: nchan " + std::to_string(nchan) +
                       " exceeds the 32768-channel limit of its fixed scratch";
        return VSPEC_ERR_UNSUPPORTED;
    }
    if (!aligned16(d_in) || !aligned16(d_accum)) return VSPEC_ERR_ALIGNMENT;
    if (nspectra == 0) return VSPEC_OK;

    int dev = 0;
    VSPEC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return VSPEC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocDevice &d = g_noalloc_dev[dev];
    if (!d.ready) {
        // once per device, with that device current: the array's device address
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        VSPEC_CUDA(cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev));
        d.base = static_cast<unsigned char *>(ptr);
        d.ready = true;
    }
    cudaStream_t st = (cudaStream_t)stream;

    NoAllocCfg c{};
    c.N = nchan;
    c.P = mode == VSPEC_PFB ? ntaps : 1;
    c.npol = npol;
    c.mode = mode;
    c.window = window;
    vspec_status r = noalloc_configure(&c, d.num_sms);
    if (r != VSPEC_OK) return r;

    float *coef = reinterpret_cast<float *>(d.base + kNaCoef);
    float2 *twA = reinterpret_cast<float2 *>(d.base + kNaTwA);
    float2 *twB = reinterpret_cast<float2 *>(d.base + kNaTwB);
    float2 *twZ = reinterpret_cast<float2 *>(d.base + kNaTwZ);
    int *kA = reinterpret_cast<int *>(d.base + kNaInts);
    int *invA = kA + kNoAllocMaxChan;
    int *invB = invA + kNoAllocMaxChan;
    void *Z = d.base + kNaZ;
    void *partial = d.base + kNaPartial;

    // The array keeps the last call's tables; rebuild them when the problem
    // changes. A rebuild enqueued into a stream capture would only run when
    // the graph is launched, while the host record below would claim the
    // tables are already there: refuse it.
    const int key[5] = {c.N, c.P, c.npol, c.mode, c.window};
    if (!d.tables_valid || std::memcmp(key, d.key, sizeof(key)) != 0) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        VSPEC_CUDA(cudaStreamIsCapturing(st, &cap));
        if (cap != cudaStreamCaptureStatusNone) {
            g_last_error = "vspec_execute_noalloc: the problem differs from the previous call's, and its "
                           "tables cannot be rebuilt inside a stream capture";
            return VSPEC_ERR_UNSUPPORTED;
        }
        d.tables_valid = false;
        const int N = c.N, Lc = c.P * N;
        vspec::gen_coef_kernel<<<(Lc + 255) / 256, 256, 0, st>>>(coef, N, Lc, mode == VSPEC_PFB ? 1 : 0, window);
        for (int i = 0; i < c.nA; i++)
            if (c.passA[i].m * (c.passA[i].r - 1) > 0)
                vspec::gen_pass_tw_kernel<<<(c.passA[i].m * (c.passA[i].r - 1) + 255) / 256, 256, 0, st>>>(twA, c.passA[i]);
        for (int i = 0; i < c.nB; i++)
            if (c.passB[i].m * (c.passB[i].r - 1) > 0)
                vspec::gen_pass_tw_kernel<<<(c.passB[i].m * (c.passB[i].r - 1) + 255) / 256, 256, 0, st>>>(twB, c.passB[i]);
        noalloc_digrev_kernel<<<(std::max(c.N1, c.N2) + 255) / 256, 256, 0, st>>>(kA, invA, invB, c.N2, c.N1, c);
        vspec::gen_twz_kernel<<<(N + 255) / 256, 256, 0, st>>>(twZ, N, c.N1, c.N2, kA);
        VSPEC_CUDA(cudaGetLastError());
        std::memcpy(d.key, key, sizeof(key));
        d.tables_valid = true;
    }

    // partial sums must start at zero on every call
    const size_t accel = npol == 2 ? sizeof(float4) : sizeof(float);
    VSPEC_CUDA(cudaMemsetAsync(partial, 0, (size_t)c.slots * c.N * accel, st));

    vspec::ColParams ca{};
    ca.in = d_in;
    ca.coef = coef;
    ca.twA = twA;
    ca.twZ = twZ;
    ca.Z = Z;
    ca.N = c.N;
    ca.N1 = c.N1;
    ca.N2 = c.N2;
    ca.C = c.C;
    ca.P = c.P;
    ca.lC = ilog2(c.C);
    ca.lN2 = ilog2(c.N2);
    ca.npass = c.nA;
    for (int i = 0; i < c.nA; i++) ca.pass[i] = c.passA[i];
    vspec::RowParams cb{};
    cb.Z = Z;
    cb.partial = partial;
    cb.twB = twB;
    cb.N = c.N;
    cb.N1 = c.N1;
    cb.N2 = c.N2;
    cb.RB = c.RB;
    cb.lN1 = ilog2(c.N1);
    cb.lRB = ilog2(c.RB);
    cb.npass = c.nB;
    for (int i = 0; i < c.nB; i++) cb.pass[i] = c.passB[i];
    cb.tiles = c.N2 / c.RB;
    cb.slots = c.slots;
    ca.tiles = c.N1 / c.C;
    ca.nframes = cb.nframes = (long long)nspectra + c.P - 1;

    const int sc_full = std::min(nspectra, c.sc_max);
    for (int s0 = 0; s0 < nspectra; s0 += sc_full) {
        const int sc = std::min(sc_full, nspectra - s0);
        ca.s0 = s0;
        ca.sc = sc;
        void *argsA[] = {&ca};
        const int ga = (int)std::min<long long>(c.blocks_a, (long long)ca.tiles * sc);
        VSPEC_CUDA(cudaLaunchKernel(c.kA, dim3(ga), dim3(c.TA), argsA, c.smemA, st));
        cb.sc = sc;
        void *argsB[] = {&cb};
        const int gb = (int)std::min<long long>(c.blocks_b, (long long)cb.tiles * sc);
        VSPEC_CUDA(cudaLaunchKernel(c.kB, dim3(gb), dim3(c.TB), argsB, c.smemB, st));
    }
    const void *part = partial;
    int groups = c.slots, stride = 1, N = c.N, N1 = c.N1, N2 = c.N2;  // at most 16 slots
    const int *ia = invA, *ib = invB;
    void *outp = d_accum;
    void *argsR[] = {&part, &groups, &stride, &N, &N1, &N2, &ia, &ib, &outp};
    VSPEC_CUDA(cudaLaunchKernel(c.kR, dim3((c.N + 31) / 32), dim3(32, 8), argsR, 0, st));
    return VSPEC_OK;
}
