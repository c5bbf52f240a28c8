// vspec_batch.cu — many banks (beams, sub-bands) channelized by one CUDA-graph launch.
//
// VEGAS runs one spectrometer pipeline per beam (§3 of arXiv 1411.0436), and
// the per-invocation launch and copy overheads dominate at small FFT lengths
// (§5). A batch owns one plan per bank; vspec_batch_execute records every
// bank's kernels into one CUDA graph, one forked stream branch per bank so
// that banks of different sizes run concurrently, and replays it with a
// single graph launch. In persistent mode (vspec_batch_set_persistent) the
// graph instead holds one cooperative launch that runs every bank's kernels
// as tickets of one kernel (vspec_bp.cuh, through vspec_internal.h); the rest
// is built on the public C ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <new>
#include <vector>

#include "vspec.h"
#include "vspec_internal.h"

struct vspec_batch {
    int nbanks = 0;
    std::vector<vspec_bank> desc;
    std::vector<vspec_plan *> plans;
    std::vector<unsigned> flags;
    std::vector<vspec_tuning> tuning;  // launch shape the autotuner chose
    std::vector<cudaStream_t> branch;
    std::vector<cudaEvent_t> joined;
    cudaStream_t capture = nullptr;
    cudaEvent_t forked = nullptr;
    cudaGraphExec_t exec = nullptr;
    // persistent mode: control words and timeout flag of the multi-bank launch
    bool persistent = false;
    int *bp_ctl = nullptr, *bp_status = nullptr;
    int stall_bank = -1;
    // arguments the graph was captured with
    std::vector<const int8_t *> g_in;
    std::vector<int> g_ns;
    std::vector<float *> g_acc;
};

namespace {

void destroy_batch(vspec_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (vspec_plan *p : b->plans) vspec_plan_destroy(p);
    for (cudaStream_t s : b->branch) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->joined) cudaEventDestroy(e);
    if (b->forked) cudaEventDestroy(b->forked);
    if (b->capture) cudaStreamDestroy(b->capture);
    cudaFree(b->bp_ctl);
    cudaFree(b->bp_status);
    delete b;
}

vspec_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return VSPEC_OK;
    return e == cudaErrorMemoryAllocation ? VSPEC_ERR_OOM : VSPEC_ERR_CUDA;
}

// Record all banks into a graph: fork from `capture` to one branch per bank,
// vspec_execute on each branch, join back.
vspec_status capture_graph(vspec_batch *b, const int8_t *const *d_in, const int *nspectra,
                           float *const *d_accum) {
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return VSPEC_ERR_CUDA;
    vspec_status st = VSPEC_OK;
    if (b->persistent) {  // one cooperative launch over every bank
        st = vspec_bp_execute(b->plans.data(), b->nbanks, d_in, nspectra, d_accum, b->bp_ctl, b->bp_status, -1,
                              b->capture);
    }
    e = cudaEventRecord(b->forked, b->capture);
    for (int i = 0; i < b->nbanks && e == cudaSuccess && st == VSPEC_OK && !b->persistent; i++) {
        e = cudaStreamWaitEvent(b->branch[i], b->forked, 0);
        if (e != cudaSuccess) break;
        st = vspec_execute(b->plans[i], d_in[i], nspectra[i], d_accum[i], (void *)b->branch[i]);
        if (st != VSPEC_OK) break;
        e = cudaEventRecord(b->joined[i], b->branch[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->capture, b->joined[i], 0);
    }
    cudaError_t e2 = cudaStreamEndCapture(b->capture, &graph);
    if (st != VSPEC_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return VSPEC_ERR_CUDA;
    }
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return VSPEC_ERR_CUDA;
    b->g_in.assign(d_in, d_in + b->nbanks);
    b->g_ns.assign(nspectra, nspectra + b->nbanks);
    b->g_acc.assign(d_accum, d_accum + b->nbanks);
    return VSPEC_OK;
}

bool same_args(const vspec_batch *b, const int8_t *const *d_in, const int *nspectra,
               float *const *d_accum) {
    if (!b->exec) return false;
    for (int i = 0; i < b->nbanks; i++)
        if (b->g_in[i] != d_in[i] || b->g_ns[i] != nspectra[i] || b->g_acc[i] != d_accum[i]) return false;
    return true;
}

}  // namespace

extern "C" {

vspec_status vspec_batch_create(vspec_batch **out, int nbanks, const vspec_bank *banks) {
    if (!out) return VSPEC_ERR_INVALID_ARG;
    *out = nullptr;
    if (nbanks < 1 || nbanks > 256 || !banks) return VSPEC_ERR_INVALID_ARG;
    vspec_batch *b = new (std::nothrow) vspec_batch();
    if (!b) return VSPEC_ERR_OOM;
    b->nbanks = nbanks;
    b->desc.assign(banks, banks + nbanks);
    b->flags.assign(nbanks, 0u);
    b->tuning.assign(nbanks, vspec_tuning{});
    for (int i = 0; i < nbanks; i++) {
        vspec_plan *p = nullptr;
        const vspec_bank &d = banks[i];
        vspec_status st = vspec_plan_create(&p, d.nchan, d.ntaps, d.npol, d.mode, d.window);
        if (st != VSPEC_OK) {
            destroy_batch(b);
            return st;
        }
        b->plans.push_back(p);
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            if (s) cudaStreamDestroy(s);
            destroy_batch(b);
            return VSPEC_ERR_CUDA;
        }
        b->branch.push_back(s);
        b->joined.push_back(e);
    }
    if (cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->forked, cudaEventDisableTiming) != cudaSuccess) {
        destroy_batch(b);
        return VSPEC_ERR_CUDA;
    }
    *out = b;
    return VSPEC_OK;
}

vspec_status vspec_batch_destroy(vspec_batch *batch) {
    destroy_batch(batch);
    return VSPEC_OK;
}

vspec_status vspec_batch_execute(vspec_batch *batch, const int8_t *const *d_in, const int *nspectra,
                                 float *const *d_accum, void *stream) {
    if (!batch || !d_in || !nspectra || !d_accum) return VSPEC_ERR_INVALID_ARG;
    for (int i = 0; i < batch->nbanks; i++) {
        if (!d_in[i] || !d_accum[i] || nspectra[i] < 0) return VSPEC_ERR_INVALID_ARG;
        if (((uintptr_t)d_in[i] & 15u) || ((uintptr_t)d_accum[i] & 15u)) return VSPEC_ERR_ALIGNMENT;
    }
    if (batch->persistent && batch->stall_bank >= 0) {  // one launch with the injected stall, outside the graph
        const int bank = batch->stall_bank;
        batch->stall_bank = -1;
        return vspec_bp_execute(batch->plans.data(), batch->nbanks, d_in, nspectra, d_accum, batch->bp_ctl,
                                batch->bp_status, bank, (cudaStream_t)stream);
    }
    if (!same_args(batch, d_in, nspectra, d_accum)) {
        vspec_status st = capture_graph(batch, d_in, nspectra, d_accum);
        if (st != VSPEC_OK) return st;
    }
    return cuda_status(cudaGraphLaunch(batch->exec, (cudaStream_t)stream));
}

vspec_status vspec_batch_autotune(vspec_batch *batch, const int8_t *const *d_in, const int *nspectra,
                                  float *const *d_accum, void *stream, int reps) {
    if (!batch || !d_in || !nspectra || !d_accum || reps < 1) return VSPEC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess) return VSPEC_ERR_CUDA;
    vspec_status result = VSPEC_OK;
    // time one plan in its current shape: a warm-up execute, then reps
    auto time_plan = [&](vspec_plan *p, int i, float *ms) -> bool {
        vspec_status s = vspec_execute(p, d_in[i], nspectra[i], d_accum[i], stream);
        cudaEventRecord(t0, st);
        for (int r = 0; r < reps && s == VSPEC_OK; r++) s = vspec_execute(p, d_in[i], nspectra[i], d_accum[i], stream);
        cudaEventRecord(t1, st);
        return s == VSPEC_OK && cudaEventSynchronize(t1) == cudaSuccess &&
               cudaEventElapsedTime(ms, t0, t1) == cudaSuccess;
    };
    for (int i = 0; i < batch->nbanks && result == VSPEC_OK; i++) {
        const vspec_bank &d = batch->desc[i];
        // plan candidates: the default plan, the two-kernel plan, and the
        // two-kernel plan with the four-step split moved one factor of two
        // either way (rows twice or half as long) and with the general
        // kernel A at twice or half the default tile width
        struct Cand {
            unsigned flags;
            int col_len, tile_cols;
        };
        std::vector<Cand> cand{{0u, 0, 0}, {VSPEC_PLAN_TWO_KERNEL, 0, 0}};
        {
            vspec_plan *probe = nullptr;
            int n2 = 0, cols = 0;
            if (vspec_plan_create_ex(&probe, d.nchan, d.ntaps, d.npol, d.mode, d.window, VSPEC_PLAN_TWO_KERNEL) ==
                VSPEC_OK) {
                vspec_plan_get_shape(probe, &n2, &cols);
                vspec_plan_destroy(probe);
            }
            if (n2 > 1) {
                cand.push_back({VSPEC_PLAN_TWO_KERNEL, n2 * 2, 0});
                cand.push_back({VSPEC_PLAN_TWO_KERNEL, n2 / 2, 0});
                cand.push_back({VSPEC_PLAN_TWO_KERNEL, n2, cols * 2});
                if (cols > 1) cand.push_back({VSPEC_PLAN_TWO_KERNEL, n2, cols / 2});
            }
        }
        float best = 1e30f;
        vspec_plan *best_plan = nullptr;
        unsigned best_flags = 0;
        vspec_tuning best_tuning{};
        for (const Cand &cd : cand) {
            const unsigned f = cd.flags;
            vspec_plan *p = nullptr;
            if (vspec_plan_create_shaped(&p, d.nchan, d.ntaps, d.npol, d.mode, d.window, f, cd.col_len,
                                         cd.tile_cols) != VSPEC_OK)
                continue;  // a shape the kernels cannot hold
            // launch shapes: the plan's default, a chunk a half and a quarter
            // as long, kernel B over two waves of CTAs, and for a fused plan
            // each path alone
            vspec_tuning def{}, lim{};
            vspec_plan_get_tuning(p, &def, &lim);
            std::vector<vspec_tuning> shapes{def};
            for (int div : {2, 4}) {
                if (def.chunk_spectra >= div) {
                    vspec_tuning t = def;
                    t.chunk_spectra = def.chunk_spectra / div;
                    shapes.push_back(t);
                }
            }
            if (def.chunk_spectra > 0 && lim.blocks_b >= 2) {
                vspec_tuning t = def;
                t.blocks_b = lim.blocks_b / 2;  // the limit is four waves
                shapes.push_back(t);
            }
            if (lim.two_kernel_from > 0) {  // a fused plan owning a two-kernel plan
                for (int from : {0, INT_MAX}) {
                    if (from == def.two_kernel_from) continue;
                    vspec_tuning t = def;
                    t.two_kernel_from = from;
                    shapes.push_back(t);
                }
            }
            bool kept = false;
            for (const vspec_tuning &t : shapes) {
                float ms = 0.f;
                if (vspec_plan_set_tuning(p, &t) != VSPEC_OK || !time_plan(p, i, &ms)) {
                    cudaStreamSynchronize(st);
                    continue;
                }
                if (ms < best) {
                    if (best_plan && best_plan != p) vspec_plan_destroy(best_plan);
                    best_plan = p;
                    best = ms;
                    best_flags = f;
                    best_tuning = t;
                    kept = true;
                }
            }
            cudaStreamSynchronize(st);
            if (!kept) vspec_plan_destroy(p);
        }
        if (!best_plan) {
            result = VSPEC_ERR_CUDA;
            break;
        }
        cudaStreamSynchronize(st);
        // a chunk longer than the bank's call is the same launch as one of the
        // call's length: keep that, and trim the scratch to it
        if (best_tuning.chunk_spectra > nspectra[i] && nspectra[i] > 0) best_tuning.chunk_spectra = nspectra[i];
        if (vspec_plan_set_tuning(best_plan, &best_tuning) != VSPEC_OK) result = VSPEC_ERR_CUDA;
        if (result == VSPEC_OK && best_tuning.chunk_spectra > 0) result = vspec_plan_trim_scratch(best_plan);
        vspec_plan_destroy(batch->plans[i]);
        batch->plans[i] = best_plan;
        batch->flags[i] = best_flags;
        batch->tuning[i] = best_tuning;
        const size_t bytes = (size_t)d.nchan * (d.npol == 2 ? 4 : 1) * sizeof(float);
        if (cudaMemsetAsync(d_accum[i], 0, bytes, st) != cudaSuccess) result = VSPEC_ERR_CUDA;
    }
    if (batch->exec) {
        cudaGraphExecDestroy(batch->exec);
        batch->exec = nullptr;
    }
    // the whole batch: per-bank kernels in one graph against one persistent
    // launch over all banks (where every bank has a ticket body); keep the faster
    if (result == VSPEC_OK) {
        auto time_batch = [&](float *ms) -> bool {
            vspec_status s = vspec_batch_execute(batch, d_in, nspectra, d_accum, stream);
            cudaEventRecord(t0, st);
            for (int r = 0; r < reps && s == VSPEC_OK; r++) s = vspec_batch_execute(batch, d_in, nspectra, d_accum, stream);
            cudaEventRecord(t1, st);
            return s == VSPEC_OK && cudaEventSynchronize(t1) == cudaSuccess &&
                   cudaEventElapsedTime(ms, t0, t1) == cudaSuccess;
        };
        float ms_graph = 0.f, ms_pers = 0.f;
        batch->persistent = false;
        const bool g_ok = time_batch(&ms_graph);
        // persistent trial: banks whose tuned plan has no ticket body run their
        // two-kernel plan in it; the tuned plans come back if the graph wins
        std::vector<vspec_plan *> tuned = batch->plans, alt = batch->plans;
        bool p_ok = g_ok && batch->nbanks <= 16;
        for (int i = 0; i < batch->nbanks && p_ok; i++) {
            if (vspec_bp_supported(tuned[i], nullptr) == VSPEC_OK) continue;
            const vspec_bank &d = batch->desc[i];
            alt[i] = nullptr;
            if (vspec_plan_create_ex(&alt[i], d.nchan, d.ntaps, d.npol, d.mode, d.window, VSPEC_PLAN_TWO_KERNEL) !=
                    VSPEC_OK ||
                vspec_bp_supported(alt[i], nullptr) != VSPEC_OK)
                p_ok = false;
        }
        if (p_ok) {
            batch->plans = alt;
            p_ok = vspec_batch_set_persistent(batch, 1) == VSPEC_OK && time_batch(&ms_pers) &&
                   vspec_batch_check(batch) == VSPEC_OK;
        }
        cudaStreamSynchronize(st);
        const bool keep = p_ok && ms_pers < ms_graph;
        for (int i = 0; i < batch->nbanks; i++) {
            if (alt[i] == tuned[i]) continue;
            if (keep) {
                vspec_plan_destroy(tuned[i]);
                batch->flags[i] = VSPEC_PLAN_TWO_KERNEL;
                vspec_plan_get_tuning(alt[i], &batch->tuning[i], nullptr);
            } else if (alt[i]) {
                vspec_plan_destroy(alt[i]);
            }
        }
        if (!keep) {
            batch->plans = tuned;
            vspec_batch_set_persistent(batch, 0);
        }
        cudaStreamSynchronize(st);
        for (int i = 0; i < batch->nbanks; i++) {
            const vspec_bank &d = batch->desc[i];
            const size_t bytes = (size_t)d.nchan * (d.npol == 2 ? 4 : 1) * sizeof(float);
            if (cudaMemsetAsync(d_accum[i], 0, bytes, st) != cudaSuccess) result = VSPEC_ERR_CUDA;
        }
        cudaStreamSynchronize(st);
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    return result;
}

vspec_status vspec_batch_bank_tuning(const vspec_batch *batch, int bank, unsigned *flags, vspec_tuning *tuning) {
    if (!batch || bank < 0 || bank >= batch->nbanks) return VSPEC_ERR_INVALID_ARG;
    if (flags) *flags = batch->flags[bank];
    if (tuning) return vspec_plan_get_tuning(batch->plans[bank], tuning, nullptr);
    return VSPEC_OK;
}

vspec_status vspec_batch_bank_shape(const vspec_batch *batch, int bank, int *col_len, int *tile_cols) {
    if (!batch || bank < 0 || bank >= batch->nbanks) return VSPEC_ERR_INVALID_ARG;
    return vspec_plan_get_shape(batch->plans[bank], col_len, tile_cols);
}

vspec_status vspec_batch_set_persistent(vspec_batch *batch, int enable) {
    if (!batch) return VSPEC_ERR_INVALID_ARG;
    if (batch->exec) {  // the next execute captures the other form
        cudaGraphExecDestroy(batch->exec);
        batch->exec = nullptr;
    }
    if (!enable) {
        batch->persistent = false;
        return VSPEC_OK;
    }
    if (batch->nbanks > 16) {
        vspec_set_last_error("the persistent launch holds at most 16 banks");
        return VSPEC_ERR_UNSUPPORTED;
    }
    // a bank whose plan has no ticket body in the kernel gets its two-kernel plan
    for (int i = 0; i < batch->nbanks; i++) {
        const char *why = nullptr;
        if (vspec_bp_supported(batch->plans[i], &why) == VSPEC_OK) continue;
        const vspec_bank &d = batch->desc[i];
        vspec_plan *p = nullptr;
        vspec_status st = vspec_plan_create_ex(&p, d.nchan, d.ntaps, d.npol, d.mode, d.window, VSPEC_PLAN_TWO_KERNEL);
        if (st != VSPEC_OK) return st;
        if (vspec_bp_supported(p, &why) != VSPEC_OK) {
            vspec_plan_destroy(p);
            vspec_set_last_error(why);
            return VSPEC_ERR_UNSUPPORTED;
        }
        vspec_plan_destroy(batch->plans[i]);
        batch->plans[i] = p;
        batch->flags[i] = VSPEC_PLAN_TWO_KERNEL;
        vspec_plan_get_tuning(p, &batch->tuning[i], nullptr);
    }
    if (!batch->bp_ctl) {
        if (cudaMalloc(&batch->bp_ctl, sizeof(int) * (2 + 2 * 16)) != cudaSuccess ||
            cudaMalloc(&batch->bp_status, sizeof(int)) != cudaSuccess ||
            cudaMemset(batch->bp_status, 0, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(batch->bp_ctl);
            cudaFree(batch->bp_status);
            batch->bp_ctl = batch->bp_status = nullptr;
            return VSPEC_ERR_OOM;
        }
    }
    batch->persistent = true;
    return VSPEC_OK;
}

vspec_status vspec_batch_get_persistent(const vspec_batch *batch, int *enabled) {
    if (!batch || !enabled) return VSPEC_ERR_INVALID_ARG;
    *enabled = batch->persistent ? 1 : 0;
    return VSPEC_OK;
}

vspec_status vspec_batch_check(vspec_batch *batch) {
    if (!batch) return VSPEC_ERR_INVALID_ARG;
    if (!batch->bp_status) return VSPEC_OK;
    int h = 0;
    if (cudaMemcpy(&h, batch->bp_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return VSPEC_ERR_CUDA;
    if (!h) return VSPEC_OK;
    if (cudaMemset(batch->bp_status, 0, sizeof(int)) != cudaSuccess) return VSPEC_ERR_CUDA;
    vspec_set_last_error("a bounded wait of the persistent multi-bank kernel gave up; results are incomplete");
    return VSPEC_ERR_DEVICE_TIMEOUT;
}

vspec_status vspec_batch_inject_stall(vspec_batch *batch, int bank) {
    if (!batch || bank < 0 || bank >= batch->nbanks) return VSPEC_ERR_INVALID_ARG;
    if (!batch->persistent) {
        vspec_set_last_error("only the persistent form waits on other CTAs' work");
        return VSPEC_ERR_UNSUPPORTED;
    }
    batch->stall_bank = bank;
    return VSPEC_OK;
}

vspec_status vspec_batch_bank_flags(const vspec_batch *batch, int bank, unsigned *flags) {
    if (!batch || bank < 0 || bank >= batch->nbanks || !flags) return VSPEC_ERR_INVALID_ARG;
    *flags = batch->flags[bank];
    return VSPEC_OK;
}

}  // extern "C"
