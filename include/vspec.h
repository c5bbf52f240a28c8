/*
 * vspec.h — C ABI of the GB300 streaming channelizer (arXiv 1411.0436).
 *
 * The library implements the GPU spectrometer of §4 of "A GPU-Based Wide-Band
 * Radio Spectrometer": 8-bit dual- or single-polarisation complex voltages
 * are pre-filtered by a P-tap polyphase filter bank (or not, in direct-FFT
 * mode, §5), transformed by an N-point FFT per polarisation, detected into
 * X^2, Y^2, Re(XY*) and Im(XY*) and accumulated over the integration (§4).
 * The initialisation steps of §4's algorithm (loading filter coefficients,
 * creating the FFT plan) map to vspec_plan_create; the processing loop
 * (pre-filter, FFTs, accumulate) maps to vspec_execute; copying the output to
 * the host maps to vspec_dump.
 *
 * Conventions (the paper leaves these unstated; they are fixed here):
 *   - input layout   int8, [time][pol][re, im]; single-pol is [time][re, im];
 *   - coefficients   h[i] = w[i] * sinc((i - (L-1)/2) / N), L = P*N, with a
 *                    symmetric window w of length L (rect, Hann or Hamming);
 *                    direct mode multiplies by the bare window of length N;
 *   - tap order      h[t*N + n] multiplies frame s+t of spectrum s;
 *   - hop            N samples (critically sampled filter bank);
 *   - DFT            X[k] = sum_n y[n] exp(-2 pi i n k / N), unnormalised,
 *                    natural channel order (k = 0 is DC);
 *   - output         npol == 2: float4 per channel (XX, YY, Re XY*, Im XY*),
 *                    XY* = X * conj(Y); npol == 1: one float (XX) per channel;
 *   - accumulation   a plain FP32 sum over spectra into the caller's buffer.
 *
 * All device pointers are plain CUDA device addresses (for example from
 * cudaMalloc or a framework's allocator); `stream` is a cudaStream_t passed as
 * void* (NULL selects the legacy default stream). No call throws; every call
 * returns a vspec_status. Calls on one plan must not run concurrently from
 * several host threads; separate plans are independent.
 */
#ifndef VSPEC_H
#define VSPEC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define VSPEC_API __attribute__((visibility("default")))
#else
#define VSPEC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VSPEC_OK = 0,
    VSPEC_ERR_INVALID_ARG = -1,    /* a size, mode, window or pointer is out of range   */
    VSPEC_ERR_UNSUPPORTED = -2,    /* a valid combination this build does not implement */
    VSPEC_ERR_ALIGNMENT = -3,      /* a device pointer is not 16-byte aligned           */
    VSPEC_ERR_CUDA = -4,           /* a CUDA runtime call or kernel launch failed       */
    VSPEC_ERR_OOM = -5,            /* device memory for the plan could not be allocated */
    VSPEC_ERR_DEVICE_TIMEOUT = -6  /* a bounded device-side wait expired                */
} vspec_status;

typedef enum { VSPEC_PFB = 0, VSPEC_DIRECT = 1 } vspec_mode;

typedef enum { VSPEC_WIN_RECT = 0, VSPEC_WIN_HANN = 1, VSPEC_WIN_HAMMING = 2 } vspec_window;

typedef struct vspec_plan vspec_plan;

/*
 * Create a plan (§4, initialisation: load the filter coefficients and create
 * the FFT plan for the polarisations processed in parallel).
 *   nchan   channels N: a power of two in [16, 2^20];
 *   ntaps   taps P: 1..16 in PFB mode; 0 or 1 in direct mode;
 *   npol    1 or 2;
 *   mode    VSPEC_PFB or VSPEC_DIRECT;
 *   window  VSPEC_WIN_RECT, VSPEC_WIN_HANN or VSPEC_WIN_HAMMING.
 * Coefficients and twiddle factors are generated on the current CUDA device in
 * FP64 and stored in FP32; the plan also owns its scratch buffers. The plan is
 * bound to the device that is current at creation. On success *out holds the
 * plan; on failure *out is set to NULL and nothing is leaked.
 * Errors: VSPEC_ERR_INVALID_ARG (bad argument or out == NULL),
 * VSPEC_ERR_OOM, VSPEC_ERR_CUDA. Every valid (nchan, ntaps, npol, mode,
 * window) is implemented; VSPEC_ERR_UNSUPPORTED comes only from the flags of
 * vspec_plan_create_ex and the sub-band limits of vspec_plan_create_sb.
 */
VSPEC_API vspec_status vspec_plan_create(vspec_plan **out, int nchan, int ntaps, int npol,
                               vspec_mode mode, vspec_window window);

/* Plan flags for vspec_plan_create_ex. */
#define VSPEC_PLAN_TWO_KERNEL 1u /* use the general two-kernel path even where the one-pass
                                    fused path applies (for comparison and testing) */
#define VSPEC_PLAN_TENSOR 2u     /* two-kernel path with DFT stages on the tensor cores;
                                    dual-pol only, nchan 2^11..2^20 where the rows are 2048
                                    points (other sizes return VSPEC_ERR_UNSUPPORTED).
                                    PFB of 5..8 taps at nchan 2^15..2^17: kernel A's whole
                                    column DFT (16, 32 or 64 points) as one tensor-core
                                    product of the fp16-rounded FIR output with the DFT
                                    matrix in fp16 hi/lo parts (two MMA terms), fp32
                                    accumulation. Other sizes and direct mode: the first
                                    radix-16 pass of every row with bf16 hi/lo operands
                                    (about 16 bits, vspec_tc_dft16). */
#define VSPEC_PLAN_TENSOR_INT8 8u /* two-kernel path whose kernel A is one tensor-core product
                                    per column on the int8 input itself (exact in fp16): the
                                    pre-filter taps and the column DFT folded into fp16
                                    coefficient matrices computed at plan time (high and low
                                    parts where they fit in shared memory), fp32
                                    accumulation. Dual-pol PFB of at most 8 taps or direct
                                    mode, nchan 2^15..2^17 (else VSPEC_ERR_UNSUPPORTED).
                                    Combinable with VSPEC_PLAN_KAHAN. */
#define VSPEC_PLAN_KAHAN 4u      /* compensated (Kahan) FP32 accumulation at every level: over
                                    spectra in the kernel, across groups and into the caller's
                                    accumulator through a plan-owned compensation buffer that
                                    vspec_dump clears; uses the two-kernel path (combinable with
                                    VSPEC_PLAN_TENSOR). With it, keep one accumulator per plan. */
#define VSPEC_PLAN_RING 16u      /* the two-kernel path as one persistent launch per call
                                    (cooperative: one CTA per SM): kernel-A and kernel-B work
                                    handed out in dependency order, the four-step intermediate
                                    in a ring of a few chunk slots (about 32 MiB each) that stays
                                    in L2 instead of going through HBM. Dual-pol PFB of 5..8
                                    taps with 2048-point rows (nchan 2^12..2^18); other plans
                                    return VSPEC_ERR_UNSUPPORTED. Its waits are bounded (see
                                    vspec_set_wait_limit; vspec_plan_check reports one that gave
                                    up). Shape: vspec_plan_set_ring. */

/*
 * vspec_plan_create with flags (a bitwise OR of VSPEC_PLAN_* values; 0 gives
 * vspec_plan_create). Unknown flag bits return VSPEC_ERR_INVALID_ARG.
 */
VSPEC_API vspec_status vspec_plan_create_ex(vspec_plan **out, int nchan, int ntaps, int npol,
                                            vspec_mode mode, vspec_window window, unsigned flags);

/*
 * vspec_plan_create_ex with an explicit shape of the two-kernel path (for the
 * batch autotuner and experiments): col_len is the column length N2 of the
 * four-step split (rows of nchan / col_len points, at most 4096), tile_cols
 * the width in columns of kernel A's tiles (which selects the general kernel
 * A); 0 keeps the plan's own choice of each. A non-zero shape implies
 * VSPEC_PLAN_TWO_KERNEL. Results agree with the default plan's within the
 * FP32 tolerance. Errors: as vspec_plan_create_ex, and VSPEC_ERR_UNSUPPORTED
 * for a shape the kernels cannot hold (the reason in vspec_last_error).
 * vspec_plan_get_shape reports a plan's col_len and tile_cols (0 for a
 * one-pass fused plan without a two-kernel plan).
 */
VSPEC_API vspec_status vspec_plan_create_shaped(vspec_plan **out, int nchan, int ntaps, int npol,
                                                vspec_mode mode, vspec_window window, unsigned flags,
                                                int col_len, int tile_cols);
VSPEC_API vspec_status vspec_plan_get_shape(const vspec_plan *plan, int *col_len, int *tile_cols);

/*
 * Plan for a sub-band mode: nsub sub-bands (1..16) of nchan channels each,
 * every one channelized like a plan of vspec_plan_create_ex. VEGAS's
 * eight-sub-band modes (§3, Table 1) run 16 FFTs in parallel: 8 sub-bands x
 * 2 polarisations (§4, initialisation). Layouts of vspec_execute and the
 * other calls on such a plan:
 *   input   int8 [(nspectra + P_eff - 1) * nchan][nsub][npol][re, im]
 *           (the sub-bands of one time sample are adjacent);
 *   output  [nsub][nchan] of float4 (npol == 2) or float (npol == 1).
 * Dual-pol plans whose kernel A is a register-column form (PFB of 5..8 taps
 * or direct mode with 2048-point rows; a fused plan's own two-kernel plan
 * counts) read each sub-band of the input in place: where the tiled fold
 * applies (nchan >= 2^15), every sub-band of a chunk runs in one kernel-A
 * and one kernel-B launch, so the input is read from HBM once; otherwise
 * sub-band after sub-band over chunks of about 32 MiB of input. Other plans
 * copy chunks of about 64 MiB of input into sub-band-contiguous order in
 * plan-owned scratch first. nsub == 1 is exactly vspec_plan_create_ex.
 */
VSPEC_API vspec_status vspec_plan_create_sb(vspec_plan **out, int nchan, int ntaps, int npol, int nsub,
                                            vspec_mode mode, vspec_window window, unsigned flags);

/*
 * Synchronise with the device and report whether a bounded device-side wait
 * of this plan's kernels expired since the last check (VSPEC_ERR_DEVICE_TIMEOUT;
 * the flag is then cleared). Plans without such waits return VSPEC_OK.
 */
VSPEC_API vspec_status vspec_plan_check(vspec_plan *plan);

/*
 * Failure-path controls, for testing how callers handle a device-side wait
 * that gives up (no GPU fault is involved in any of them).
 *
 * vspec_set_wait_limit sets, for every later launch in the process, how many
 * times a kernel polls before a bounded wait for its results gives up and
 * raises the plan's timeout flag (reported by vspec_plan_check or as
 * VSPEC_ERR_DEVICE_TIMEOUT by vspec_tc_dft16): polls >= 0 sets the limit (0
 * gives up at once), polls < 0 restores the default of 2^24 (a ring kernel
 * sleeps about 100 ns between polls; when one of its waits gives up, the
 * others return at once and the launch ends). The wait that
 * drains outstanding tensor-core work before a kernel frees its tensor
 * memory always keeps the default bound. Results computed under a wait that
 * gave up are incomplete and must be discarded.
 * Errors: VSPEC_ERR_INVALID_ARG (polls above 2^32 - 1).
 *
 * vspec_plan_inject_timeout raises the plan's timeout flag from the host, as
 * if a device-side wait had expired; the next vspec_plan_check reports
 * VSPEC_ERR_DEVICE_TIMEOUT and clears it. Synchronous.
 * Errors: VSPEC_ERR_INVALID_ARG, VSPEC_ERR_UNSUPPORTED (a plan without
 * bounded device-side waits), VSPEC_ERR_CUDA.
 */
VSPEC_API vspec_status vspec_set_wait_limit(long long polls);

/*
 * Bounds checks of the debug build. The library built with -DVSPEC_DEBUG
 * (libvspec_debug.so) checks, before every access of the chunk scratch, the
 * partial-sum slots and the input frames, that the index lies inside the
 * buffer the plan or the call owns; a failed check sets a bit of a device
 * status word and the access is skipped (no trap). Bits: 1 chunk-scratch
 * index, 2 input frame, 4 partial-sum slot, 8 tile index.
 * vspec_debug_flags synchronises the device, writes that word to *flags and,
 * if clear != 0, resets it. The release build returns VSPEC_ERR_UNSUPPORTED.
 * Errors: VSPEC_ERR_INVALID_ARG, VSPEC_ERR_CUDA, VSPEC_ERR_UNSUPPORTED.
 */
VSPEC_API vspec_status vspec_debug_flags(unsigned *flags, int clear);
VSPEC_API vspec_status vspec_plan_inject_timeout(vspec_plan *plan);

/*
 * For ring plans (VSPEC_PLAN_RING): the next launch starts the done counter of
 * ring slot `slot` (counted from the call's first slot) one below zero, so
 * that slot's kernel-B tickets wait for a kernel-A ticket that never comes:
 * their bounded wait gives up, the launch ends without finishing the call,
 * and vspec_plan_check reports VSPEC_ERR_DEVICE_TIMEOUT. Applies to one launch.
 * Errors: VSPEC_ERR_INVALID_ARG, VSPEC_ERR_UNSUPPORTED (not a ring plan).
 */
VSPEC_API vspec_status vspec_plan_inject_stall(vspec_plan *plan, int slot);

/* Release a plan and all device memory it owns. NULL is accepted. The caller
 * must make sure no work using the plan is still running on any stream. */
VSPEC_API vspec_status vspec_plan_destroy(vspec_plan *plan);

/*
 * Channelize nspectra spectra and add them to d_accum (§4, processing loop:
 * pre-filter, parallel FFTs, accumulate).
 *   d_in     device int8 [(nspectra + P_eff - 1) * nchan][npol][2], P_eff = ntaps
 *            in PFB mode and 1 in direct mode; spectrum s uses samples
 *            [s*nchan, (s + P_eff)*nchan). A streaming caller overlaps
 *            consecutive calls' inputs by (P_eff - 1) * nchan samples.
 *   nspectra number of spectra, >= 0 (0 is a no-op).
 *   d_accum  device float[nchan * 4] (npol == 2, float4 per channel) or
 *            float[nchan] (npol == 1); accumulated into, never cleared here.
 *   stream   cudaStream_t (as void*) on which all work is enqueued.
 * Both pointers must be 16-byte aligned. The call is asynchronous: it returns
 * once the work is enqueued; the caller owns d_in and d_accum and must keep
 * them alive until the stream reaches the end of this call's work.
 * Errors: VSPEC_ERR_INVALID_ARG (NULL plan/pointer, nspectra < 0),
 * VSPEC_ERR_ALIGNMENT, VSPEC_ERR_CUDA (launch failure; the plan stays usable).
 */
VSPEC_API vspec_status vspec_execute(vspec_plan *plan, const int8_t *d_in, int nspectra,
                           float *d_accum, void *stream);

/*
 * The whole loop of §4 from host memory: copy the time series to the device,
 * pre-filter, FFT, detect and accumulate, and copy the output to the host,
 * with the copies overlapped with the compute through CUDA streams (the
 * pipelining §6 proposes).
 *   h_in   host int8, layout and size as d_in of vspec_execute. Pinned
 *          memory (cudaHostAlloc / cudaHostRegister) lets copies overlap
 *          compute; pageable memory works but serialises.
 *   h_out  host float[nchan * 4] (npol == 2) or float[nchan]: overwritten
 *          with the accumulated spectra of these nspectra spectra.
 * Two ways to bring the input over, chosen by vspec_plan_set_host_mode:
 *   staged  chunks of input (by default a sixteenth of the first call's input,
 *           within 32 .. 256 MiB; settable): a plan-owned copy stream fills
 *           one of two device staging buffers while a plan-owned compute
 *           stream channelizes the other;
 *   mapped  pinned host memory that the device can address (any cudaHostAlloc
 *           or cudaHostRegister buffer on a unified-address system) is read
 *           by the kernels directly, once per byte, over the host link: no
 *           staging copy at all.
 * Auto maps when cudaPointerGetAttributes reports h_in as pinned host memory
 * with a device address, and stages otherwise. The default is staged: on
 * GB300 both ways are bound by the host link (about 210 GB/s host to
 * device), staged a little faster on short calls. All work starts
 * after the work already queued on `stream`, and `stream` waits for the final
 * copy, so the caller synchronises `stream` before reading h_out. The first
 * call on a plan allocates the staging buffers (two chunks of input plus one
 * accumulator) and creates the streams. Calls on one plan must be serialised.
 * Errors: VSPEC_ERR_INVALID_ARG (also: mapped mode with an h_in the device
 * cannot address), VSPEC_ERR_ALIGNMENT (mapped h_in not 16-byte aligned),
 * VSPEC_ERR_OOM, VSPEC_ERR_CUDA.
 */
VSPEC_API vspec_status vspec_execute_host(vspec_plan *plan, const int8_t *h_in, int nspectra,
                                          float *h_out, void *stream);

#define VSPEC_HOST_AUTO 0   /* map pinned device-addressable input, else stage */
#define VSPEC_HOST_STAGED 1 /* always copy through the staging buffers */
#define VSPEC_HOST_MAPPED 2 /* always read the host input directly */

/*
 * Select how vspec_execute_host brings the input over (VSPEC_HOST_*), and the
 * staged mode's chunk: chunk_bytes of input per staging buffer, 1 MiB .. 4 GiB,
 * 0 for automatic (a sixteenth of the first call's input, within 32 .. 256
 * MiB, fixed from then on). Each chunk pays the per-call fixed costs and the
 * pipeline exposes one chunk's copy and one chunk's compute, so long calls gain
 * from longer chunks (measured on GB300 with 2.15 GB per call: 46 GHz at
 * 32 MiB, 49 GHz at 128 MiB; with 132 MB per call 32 MiB is best). A new
 * chunk size releases the staging buffers (after synchronising the device);
 * the next call allocates them again.
 * Errors: VSPEC_ERR_INVALID_ARG.
 */
VSPEC_API vspec_status vspec_plan_set_host_mode(vspec_plan *plan, int mode, size_t chunk_bytes);

/*
 * Dump the accumulator (§4, "copy output to host") and clear it.
 *   h_out  host buffer of nchan * (npol == 2 ? 4 : 1) floats, or NULL to clear
 *          only. Pinned host memory makes the copy asynchronous; with pageable
 *          memory the copy completes before the call returns.
 * Enqueues on `stream`: a device-to-host copy of d_accum into h_out (if not
 * NULL), then a clear of d_accum to zero. The caller synchronises the stream
 * before reading h_out.
 * Errors: VSPEC_ERR_INVALID_ARG, VSPEC_ERR_ALIGNMENT, VSPEC_ERR_CUDA.
 */
VSPEC_API vspec_status vspec_dump(vspec_plan *plan, float *d_accum, float *h_out, void *stream);

/*
 * Plan properties: bytes of device scratch the plan owns (coefficients,
 * twiddles and intermediate buffers) and the number of HBM passes the design
 * makes per execute: 1 when every input byte is fetched from HBM once and
 * everything else stays on chip or in L2 (overlapping PFB frames are re-read
 * from on-chip storage or L2); 2 when, in addition, the two-kernel path's
 * chunk scratch (complex FP32 per channel and spectrum) is larger than half
 * the L2 and makes a round trip through HBM. Either output pointer may be NULL.
 */
VSPEC_API vspec_status vspec_plan_info(const vspec_plan *plan, size_t *scratch_bytes, int *hbm_passes);

/*
 * The plan's decomposition and kernels as one line of text, for logs and
 * tests, e.g. "two-kernel N1=2048 N2=16 C=32 A=colreg B=row2048 chunk=2048".
 * Words:
 *   fused K=<cluster CTAs>   the one-pass cluster kernel, then " | " and the
 *                            two-kernel plan it switches to
 *   two-kernel               the general path
 *   A=colreg|coldir|general|gather|none   kernel A's form: register columns
 *                            (dual-pol PFB), register columns (dual-pol
 *                            direct), the general kernel, taps read from the
 *                            input; none for one-row transforms
 *   B=row2048|general|tensor kernel B's form
 *   fir-in-B                 one-row transform: the FIR runs in kernel B
 *   kahan                    compensated accumulation
 * Writes at most len bytes including the terminating NUL (truncating).
 * Errors: VSPEC_ERR_INVALID_ARG (plan or buf NULL, len 0).
 */
VSPEC_API vspec_status vspec_plan_describe(const vspec_plan *plan, char *buf, size_t len);

/*
 * Instrumentation. With profiling enabled, vspec_execute records a pair of
 * CUDA events on its stream around every kernel it launches; with it
 * disabled (the default) no event is recorded. Enabling or disabling clears
 * the records.
 */
VSPEC_API vspec_status vspec_plan_set_profiling(vspec_plan *plan, int enable);

/*
 * Per-kernel totals of the records made since profiling was enabled (or
 * since the last read with reset != 0): for kernel kind `kind` (0-based; a
 * kind past the last returns VSPEC_ERR_INVALID_ARG), its name, the number
 * of launches, the spectra those launches processed and the summed
 * event-measured duration in milliseconds. Reading waits for the recorded
 * events to complete. Any output pointer may be NULL.
 */
VSPEC_API vspec_status vspec_plan_kernel_stats(vspec_plan *plan, int kind, int reset,
                                               const char **name, long long *launches,
                                               long long *spectra, double *total_ms);

/*
 * Launch shape of a plan. The results do not depend on it beyond FP32
 * summation order.
 *
 * The two-kernel path (every plan but the one-pass fused one, and the
 * two-kernel plan a fused plan owns) runs the four-step FFT through a chunk
 * scratch. A chunk is a run of spectra whose column DFTs (kernel A) all
 * finish before their row DFTs (kernel B) start. Each launch splits its
 * (tile, spectrum) items evenly over its CTAs; a CTA that starts a run of a
 * column tile re-reads ntaps-1 frames to fill its FIR window, and each CTA of
 * kernel B keeps its row tile's sums in a partial-sum slot that is folded into
 * d_accum once per execute.
 *   chunk_spectra    1 .. limit.chunk_spectra (a chunk longer than the
 *                    scratch holds grows the scratch: the call then
 *                    synchronises the device and allocates); 0 for a fused
 *                    plan that owns no two-kernel plan
 *   blocks_a         CTAs per kernel-A launch: 0 (one wave, the default) or
 *                    1 .. limit.blocks_a
 *   blocks_b         CTAs per kernel-B launch: 0 (one wave) or 1 .. limit.blocks_b
 * One-pass fused plans (dual-pol, 2048..32768 channels) run clusters of CTAs.
 * Except at 2048 channels they own a two-kernel plan of the same problem,
 * which the three fields above tune, and use it in two ways:
 *   two_kernel_from  a call with at least this many spectra runs wholly on
 *                    the two-kernel path (faster on long calls: its work is
 *                    spread over every SM); 0 .. INT_MAX, INT_MAX: never. The
 *                    default is a per-size crossover measured on GB300.
 *                    Plans without a two-kernel plan: INT_MAX; two-kernel
 *                    plans: 0.
 *   assist_permille  on shorter calls, the two-kernel plan channelizes the
 *                    last assist_permille thousandths of the spectra on a
 *                    second stream, on the SMs the clusters leave idle (none
 *                    if that share is under 32 spectra): 0 .. limit (0 where
 *                    the device leaves fewer than 24 SMs idle).
 * vspec_plan_get_tuning fills the current shape and the limits (either
 * pointer may be NULL). vspec_plan_set_tuning takes effect at the next
 * execute; do not call it while an execute of the plan is in flight or being
 * captured. Errors: VSPEC_ERR_INVALID_ARG (NULL, or a value out of range),
 * VSPEC_ERR_OOM, VSPEC_ERR_CUDA (growing the scratch).
 */
typedef struct {
    int chunk_spectra;
    int blocks_a;
    int blocks_b;
    int assist_permille;
    int two_kernel_from;
} vspec_tuning;

VSPEC_API vspec_status vspec_plan_get_tuning(const vspec_plan *plan, vspec_tuning *current,
                                             vspec_tuning *limit);
VSPEC_API vspec_status vspec_plan_set_tuning(vspec_plan *plan, const vspec_tuning *tuning);

/*
 * Shrink the chunk scratch to the current chunk_spectra (it is allocated at
 * plan creation for the longest default chunk, up to 4 GiB, and only grows
 * with vspec_plan_set_tuning). Synchronises the device, then frees and
 * allocates; vspec_plan_info reports the new size. A caller whose calls are
 * shorter sets chunk_spectra to its call length and trims; the batch
 * autotuner does this for every bank. Errors: VSPEC_ERR_INVALID_ARG,
 * VSPEC_ERR_OOM (the plan then has no scratch until a tuning grows it),
 * VSPEC_ERR_CUDA.
 */
VSPEC_API vspec_status vspec_plan_trim_scratch(vspec_plan *plan);

/*
 * Shape of a VSPEC_PLAN_RING plan's persistent launch (0 keeps a value):
 *   slot_spectra  spectra per ring slot S (even, 2 .. 1024; default: the
 *                 slot nearest 32 MiB of intermediate, 16 spectra at 2^17);
 *   ring_slots    slots R of the ring (1 .. 16, at least lookahead; default 3);
 *   lookahead     slots L of kernel-A work handed out ahead of kernel-B work
 *                 (1 .. 15; default 2);
 *   row_parts     kernel-B tickets V per row tile and slot (S / V even and at
 *                 most 32; default S / 16, at least 1).
 * Kernel-B tickets sum their spectra into partial-sum sets (c mod K) V + v,
 * K = clamp(ceil(slots / 32), 2, sets / V), which a fold adds in order: the
 * result does not depend on the order in which CTAs run (it is bitwise
 * reproducible for a given shape and call length). Synchronises the device, then reallocates
 * the ring (R S nchan 16 bytes) and the sets (up to 16 MiB); vspec_plan_info
 * reports the size. Errors: VSPEC_ERR_INVALID_ARG (a value out of range),
 * VSPEC_ERR_UNSUPPORTED (not a ring plan), VSPEC_ERR_OOM, VSPEC_ERR_CUDA.
 * vspec_plan_get_ring reports the current shape (any pointer may be NULL).
 */
VSPEC_API vspec_status vspec_plan_set_ring(vspec_plan *plan, int slot_spectra, int ring_slots, int lookahead,
                                           int row_parts);
VSPEC_API vspec_status vspec_plan_get_ring(const vspec_plan *plan, int *slot_spectra, int *ring_slots,
                                           int *lookahead, int *row_parts);

/*
 * Allocation-free variant of vspec_execute. The paper has no counterpart: it
 * is for callers that cannot call cudaMalloc, such as a host application that
 * owns every byte of device memory through its own pool, or a real-time
 * capture loop in which an allocation (which can synchronise the whole
 * device) would stall the data path and drop samples.
 *
 * It channelizes the same problem as a plan created with the same (nchan,
 * ntaps, npol, mode, window), accumulating into d_accum with the same input
 * and output layouts, and gives the same result as vspec_execute within the
 * FP32 tolerance (not bit for bit: it always runs the generic two-kernel form
 * of the path, in short chunks, where a plan picks faster kernel forms). It
 * allocates nothing: coefficients, twiddles, chunk scratch and partial sums
 * live in one fixed 20 MiB device array inside this library, which every GPU
 * that loads the library holds until the process exits. Limits: nchan <=
 * 32768 (larger sizes return VSPEC_ERR_UNSUPPORTED with the reason in
 * vspec_last_error); all other arguments and errors are as for
 * vspec_plan_create and vspec_execute.
 *
 * The first call on a device (with that device current) looks up the
 * array's device address and sets kernel attributes; make that first call
 * before any stream capture. A call whose (nchan, ntaps, npol, mode, window)
 * differs from the previous call on that device rebuilds the tables in the
 * array on `stream`; such a call made while `stream` is being captured
 * returns VSPEC_ERR_UNSUPPORTED (the rebuild would only run at graph launch). Every call shares the array, which keeps the last
 * call's contents, so calls that overlap on the GPU race: serialise them
 * (one stream, or synchronise between calls). Host threads are serialised by
 * an internal lock.
 */
VSPEC_API vspec_status vspec_execute_noalloc(const int8_t *d_in, int nchan, int ntaps, int npol,
                                             vspec_mode mode, vspec_window window, int nspectra,
                                             float *d_accum, void *stream);

/*
 * Batches: many banks (beams or sub-bands, §3 runs one pipeline per beam) of
 * possibly different sizes and modes, channelized by one CUDA-graph launch.
 * A batch owns one plan per bank. The first vspec_batch_execute (and any
 * later call whose pointers or spectrum counts differ from the previous one)
 * records every bank's kernels into a CUDA graph, one forked stream branch
 * per bank so that banks run concurrently; other calls replay that graph with
 * a single launch on `stream`. Each bank follows the conventions of
 * vspec_execute for its own input and accumulator. Do not call
 * vspec_batch_execute while `stream` is being captured.
 */
typedef struct {
    int nchan;            /* as vspec_plan_create */
    int ntaps;
    int npol;
    vspec_mode mode;
    vspec_window window;
} vspec_bank;

typedef struct vspec_batch vspec_batch;

/* Create a batch of nbanks (1..256) banks. Errors as vspec_plan_create. */
VSPEC_API vspec_status vspec_batch_create(vspec_batch **out, int nbanks, const vspec_bank *banks);

/* Release a batch and its plans. NULL is accepted. */
VSPEC_API vspec_status vspec_batch_destroy(vspec_batch *batch);

/*
 * Channelize every bank: d_in[i], nspectra[i], d_accum[i] are bank i's
 * arguments of vspec_execute (host arrays of nbanks entries; the pointers they
 * hold are device pointers). Asynchronous on `stream`.
 * Errors: VSPEC_ERR_INVALID_ARG, VSPEC_ERR_ALIGNMENT, VSPEC_ERR_CUDA.
 */
VSPEC_API vspec_status vspec_batch_execute(vspec_batch *batch, const int8_t *const *d_in,
                                           const int *nspectra, float *const *d_accum, void *stream);

/*
 * Autotuner: for each bank, time `reps` executions (after one warm-up) of
 * every candidate on the given arguments and keep the fastest. Plan
 * candidates: the default plan, the two-kernel plan (VSPEC_PLAN_TWO_KERNEL),
 * and the two-kernel plan with its four-step split moved one factor of two
 * either way and with the general kernel A at twice or half its tile width
 * (vspec_plan_create_shaped). Each in several launch shapes
 * (vspec_plan_set_tuning): its default, chunks a half and a quarter as long,
 * kernel B over two waves of CTAs, and for a plan that can switch between the
 * fused and the two-kernel path, each path alone. Then the whole batch: its
 * graph of per-bank kernels against the persistent launch over all banks
 * (vspec_batch_set_persistent; banks whose chosen plan has no ticket body run
 * their two-kernel plan in it), keeping the faster (vspec_batch_get_persistent
 * reports which). Clears every d_accum[i] afterwards and synchronises `stream`. vspec_batch_bank_flags reports the
 * VSPEC_PLAN_* flags of the plan chosen for bank `bank`;
 * vspec_batch_bank_tuning also its launch shape and vspec_batch_bank_shape its
 * split and tile width (vspec_plan_get_shape); output pointers may be NULL.
 */
VSPEC_API vspec_status vspec_batch_autotune(vspec_batch *batch, const int8_t *const *d_in,
                                            const int *nspectra, float *const *d_accum,
                                            void *stream, int reps);
VSPEC_API vspec_status vspec_batch_bank_flags(const vspec_batch *batch, int bank, unsigned *flags);
VSPEC_API vspec_status vspec_batch_bank_tuning(const vspec_batch *batch, int bank, unsigned *flags,
                                               vspec_tuning *tuning);
VSPEC_API vspec_status vspec_batch_bank_shape(const vspec_batch *batch, int bank, int *col_len, int *tile_cols);

/*
 * Persistent mode: the batch's graph holds one cooperative launch (one
 * 512-thread CTA per SM) instead of every bank's kernels. That kernel runs
 * all banks' work as tickets in three phases, handed out in order by an
 * atomic counter: kernel-A tiles of every bank (the register-column forms,
 * into the bank's chunk scratch), then row tickets (32 spectra of one
 * 2048-point row, or of a one-row transform with its pre-filter), then fold
 * tickets (512 channels: the row tickets' sums, added in order and
 * compensated, into the caller's accumulator). A bank's row tickets wait
 * (bounded, vspec_set_wait_limit) until its kernel-A tickets are done, its
 * folds until its row tickets are; results do not depend on which CTA ran
 * what. A bank with a fused one-pass plan runs the two-kernel plan that the
 * fused plan owns; enabling the mode gives every other bank whose plan has no
 * ticket body its VSPEC_PLAN_TWO_KERNEL plan. Banks must be dual-pol: PFB of 5..8 taps up to
 * 2^18 channels, direct mode up to 2^19 channels, or one-row transforms
 * (up to 1024 channels with at most 8 taps, or 2048); at most 16 banks, each
 * call no longer than its plan's chunk scratch (the autotuner's choice, or
 * the default chunk). Errors of vspec_batch_set_persistent:
 * VSPEC_ERR_INVALID_ARG, VSPEC_ERR_UNSUPPORTED (a bank or the bank count;
 * the reason in vspec_last_error), VSPEC_ERR_OOM; of vspec_batch_execute in
 * this mode also VSPEC_ERR_UNSUPPORTED (a call too long for its plan).
 * enable = 0 returns to per-bank kernels. vspec_batch_autotune chooses the
 * mode by timing both.
 *
 * vspec_batch_check synchronises and reports (once) whether a wait of the
 * persistent kernel gave up (VSPEC_ERR_DEVICE_TIMEOUT; the call's results are
 * incomplete). vspec_batch_inject_stall makes the next persistent execute
 * start bank `bank`'s kernel-A done counter one below zero, so that its row
 * tickets' wait gives up (failure-path tests; no GPU fault is involved).
 */
VSPEC_API vspec_status vspec_batch_set_persistent(vspec_batch *batch, int enable);
VSPEC_API vspec_status vspec_batch_get_persistent(const vspec_batch *batch, int *enabled);
VSPEC_API vspec_status vspec_batch_check(vspec_batch *batch);
VSPEC_API vspec_status vspec_batch_inject_stall(vspec_batch *batch, int bank);

/*
 * Batched 16-point DFTs on the tensor cores (tcgen05.mma, bf16 operands,
 * fp32 accumulation in tensor memory): y[b][k] = sum_n x[b][n] exp(-2 pi i n k
 * / 16) for b < batch, the radix-16 stage of §4's FFT as a dense contraction.
 *   d_x, d_y  device complex float [batch][16] (re, im interleaved);
 *   terms     1: bf16 operands (about 8 significant bits); 3: hi/lo split of
 *             both operands, X_hi F_hi + X_hi F_lo + X_lo F_hi (about 16 bits).
 * Synchronises `stream` before returning. Errors: VSPEC_ERR_INVALID_ARG,
 * VSPEC_ERR_ALIGNMENT, VSPEC_ERR_CUDA, VSPEC_ERR_DEVICE_TIMEOUT (the bounded
 * wait for the tensor cores gave up).
 */
VSPEC_API vspec_status vspec_tc_dft16(const float *d_x, float *d_y, int batch, int terms, void *stream);

/* Static, human-readable text for a status code. */
VSPEC_API const char *vspec_status_string(vspec_status status);

/* Text of the most recent CUDA error seen by this library in the calling
 * thread ("" if none). The pointer stays valid until the thread's next call. */
VSPEC_API const char *vspec_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* VSPEC_H */
