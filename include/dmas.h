/*
 * dmas.h -- C ABI of the B300 (sm_103a) n-th order Delay-Multiply-and-Sum
 * beamformer with Coherence Factor weighting and envelope detection.
 *
 * Method: W. Jansen, W. Daems, J. Steckel, "Delay-Multiply-And-Sum Beamforming
 * for Real-Time In-Air Acoustic Imaging".  Section and equation names below
 * are that paper's.
 *
 *   For every steering direction psi and output sample t the library
 *     1. pre-steers: x_i = m_i(t + tau_{i,psi})                 (Eq. signal_delay)
 *     2. takes signed n-th roots s_i = sgn(x_i)|x_i|^(1/n)      (Sec. II-B)
 *     3. accumulates the power sums P_k = sum_i s_i^k, k=1..n  (Eq. power_sum)
 *        and sum_i x_i, sum_i x_i^2 for the coherence factor
 *     4. forms E_n from the power sums by Newton-Girard        (Eqs. dmas2_impl..
 *                                                               dmas5_impl,
 *                                                               girard_newton_general)
 *     5. weights by CF = (sum x_i)^2 / (N sum x_i^2 + eps)      (Eq. cf, Sec. II-D)
 *     6. takes |.| and low-pass filters along t (envelope)      (Sec. II, step 3)
 *   and writes image[psi][t].
 *
 * Conventions shared by every entry point:
 *   - Every call returns a dmas_status and never aborts, traps or exits.
 *   - "device" pointers are CUDA device (or managed) memory on the device that
 *     was current when the plan was created; "host" pointers are ordinary host
 *     memory.  The caller owns every buffer it passes; the library never frees
 *     or retains caller pointers beyond the call.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  Device work is enqueued asynchronously on that stream.
 *   - Sizes are element counts unless the name says bytes.
 *   - Frame values are not checked: a NaN or Inf sample propagates to the
 *     pixels that read it.
 */
#ifndef DMAS_H
#define DMAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DMAS_OK = 0,
    DMAS_EINVAL = 1,   /* a NULL, out-of-range size, order, mode or non-finite parameter */
    DMAS_ENOMEM = 2,   /* a device or host allocation failed */
    DMAS_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed (see dmas_plan_last_error) */
    DMAS_EBUSY = 4,    /* reserved for the serving layer: no capacity right now */
    DMAS_ETIMEOUT = 5, /* a device-side bounded wait expired (error word set by a kernel) */
    DMAS_EBOUNDS = 6   /* host-checked build (libdmas_checked.so) only: a kernel index fell
                          outside its buffer and the access was skipped (a library bug) */
} dmas_status;

/* How tau_{i,psi} * fs is turned into a sample position (Eq. signal_delay). */
typedef enum {
    DMAS_DELAY_ROUND = 0,  /* nearest sample, ties away from zero */
    DMAS_DELAY_LINEAR = 1  /* every power channel linearly interpolated between
                              floor(delta) and floor(delta) + 1 */
} dmas_delay_mode;

/* Storage type of the per-microphone root channel that the beamform kernel
 * gathers.  Power sums always accumulate in FP32. */
typedef enum {
    DMAS_CH_F32 = 0,
    DMAS_CH_F16 = 1,   /* roots stored as FP16 (halves the gather bytes) */
    DMAS_CH_BF16 = 2   /* roots stored as BF16 */
} dmas_chan_prec;

/* Arithmetic of the Newton-Girard step (power sums -> E_n), the one step of
 * the path whose alternating-sign cancellation needs more than FP32
 * (Sec. II-C).  The default (zero) is compensated FP32. */
typedef enum {
    DMAS_NG_CF32 = 0,  /* compensated FP32: orders <= 5 by the compensated Horner
                          scheme over Eqs. dmas2_impl..dmas5_impl, higher orders by
                          the recurrence in double-float; as accurate as the same
                          evaluation in twice FP32's precision, then rounded */
    DMAS_NG_F64 = 1,   /* FP64 (B300's FP64 rate is a small fraction of FP32's) */
    DMAS_NG_F32 = 2    /* plain FP32: a faster variant, not the default */
} dmas_ng_prec;

/* dmas_plan_desc.flags */
enum {
    DMAS_F_CF = 1,        /* multiply by the coherence factor (Eq. cf) */
    DMAS_F_ENVELOPE = 2   /* |.| then low-pass along t; without it image = E_n (x CF) */
};

typedef struct dmas_plan dmas_plan;

/*
 * Plan description.  All pointers are HOST memory, read during
 * dmas_plan_create only (the plan keeps its own copies).
 *
 * Geometry (Sec. II, delay look-up table): with delays_s == NULL the plan
 * computes tau_{i,psi} = -((p_i - p_bar) . u_psi) / c in FP64, p_bar the mean of
 * the microphone positions, u_psi the unit vector of direction psi.  The array
 * frame has x horizontal, y vertical and broadside along +z; a direction given
 * as (azimuth theta, elevation phi) is u = (sin th cos ph, sin ph, cos th cos ph)
 * (Fig. 1's azimuth/elevation).
 */
typedef struct {
    int n_mics;               /* N, 1 .. 4096 */
    const double *mic_xyz;    /* [N][3] metres; required unless delays_s is given */
    int n_dirs;               /* M, 1 .. 1<<20 */
    const double *dir_azel;   /* [M][2] radians (azimuth, elevation), or NULL */
    const double *dir_unit;   /* [M][3] unit vectors; used instead of dir_azel if non-NULL */
    const double *delays_s;   /* optional [M][N] seconds; overrides the geometry */
    int n_samples;            /* T, samples per microphone per frame, 1 .. 1<<24 */
    double fs;                /* sample rate, Hz, finite and > 0 */
    double c;                 /* speed of sound, m/s, finite and > 0 (geometry only) */
    int order;                /* n, 1 .. 8 */
    int delay_mode;           /* dmas_delay_mode */
    int flags;                /* DMAS_F_* */
    double cf_eps;            /* CF denominator constant (Eq. cf); <= 0 selects 1e-30 */
    double env_cutoff_hz;     /* envelope low-pass cutoff; <= 0 selects 5000 Hz */
    int env_taps;             /* odd FIR length <= 1023; 0 selects 2*ceil(fs/fc)+1 */
    int chan_prec;            /* dmas_chan_prec */
    int ng_prec;              /* dmas_ng_prec */
    /* Optional matched filter (Sec. II step 1, pulse compression): the emitted
     * signal e[0..mf_len-1] at fs.  Each microphone signal is replaced by its
     * correlation with e, mf_i(t) = sum_k e[k] m_i(t + k) (zero past the frame
     * end, so an echo peaks at its arrival time), before the roots.  NULL and
     * 0 turn it off; otherwise 1 <= mf_len <= 8192 and every value finite. */
    const float *mf_signal;
    int mf_len;
} dmas_plan_desc;

/* Read-only summary of a plan. */
typedef struct {
    int n_mics, n_dirs, n_samples, order, delay_mode, flags;
    int chan_prec, ng_prec;
    int env_taps;              /* L actually used (0 without DMAS_F_ENVELOPE) */
    int n_groups;              /* direction groups (CTA rows) */
    int group_size;            /* directions per group */
    int window;                /* staged samples per microphone per time tile */
    int mic_chunk;             /* microphones staged per pass */
    int time_tile;             /* output samples per CTA */
    int row;                   /* samples per root-channel row (zero pads included) */
    size_t workspace_bytes;    /* device scratch a beamform call uses */
    size_t table_bytes;        /* device bytes of the resident delay tables */
} dmas_plan_info;

/*
 * Create a plan: validates `desc`, computes the delay table in FP64, groups
 * neighbouring directions, computes the envelope taps, and allocates and
 * uploads every device table and the scratch a beamform call needs, on the
 * current CUDA device.  On success *out owns all of it.
 * Errors: DMAS_EINVAL (bad desc or out == NULL), DMAS_ENOMEM, DMAS_ECUDA.
 * On error *out is set to NULL and nothing is leaked.
 */
dmas_status dmas_plan_create(const dmas_plan_desc *desc, dmas_plan **out);

/* Release a plan and all its device memory.  NULL is a no-op returning DMAS_OK.
 * Synchronises the device before freeing. */
dmas_status dmas_destroy(dmas_plan *plan);

/*
 * Beamform one frame (the whole path, steps 1-6 above).
 *   d_frame : device [N][T] float32, row-major (microphone-major).
 *   d_image : device [M][T] float32, row-major, direction order of the desc;
 *             the envelope, or E_n (x CF) when DMAS_F_ENVELOPE is off.
 *   d_y     : optional device [M][T] float32: E_n (x CF) before the envelope.
 *   d_cf    : optional device [M][T] float32: the coherence factor.
 * The plan's scratch is reused by every call: calls on one plan must be
 * ordered on one stream (or synchronised); use one plan per concurrent stream.
 * The call only enqueues kernels on `stream` (no allocation, no
 * synchronisation, stage profiling off), so it can be captured into a CUDA
 * graph; a replay reads whatever d_frame then holds and reuses the plan's
 * scratch, under the same ordering rule.
 * Errors: DMAS_EINVAL (NULL plan/frame/image), DMAS_ECUDA (launch failure).
 * Device-side wait timeouts surface as DMAS_ETIMEOUT from dmas_plan_check.
 */
dmas_status dmas_beamform(dmas_plan *plan, const float *d_frame, float *d_image,
                          float *d_y, float *d_cf, void *stream);

/* dmas_beamform_orders: which image(s) per selected order */
enum {
    DMAS_V_PLAIN = 1,  /* E_k */
    DMAS_V_CF = 2      /* E_k x CF */
};

/*
 * Every order at once: DAS and DMAS-2..n, each with and without the coherence
 * factor (the algorithms Table I and Fig. 5 compare), from one pass over the
 * delayed samples.  The root step writes sgn(m)|m|^(1/q) for every
 * q = 1..order (Sec. II-B); the beamform step keeps per pixel sum x, sum x^2,
 * sum |x| and the power sums P_1..P_{q-1} of every q (Eq. power_sum), with
 * P_k = sum x for odd k and P_k = sum |x| for even k, and forms E_k of every
 * selected k by Newton-Girard (Eqs. dmas2_impl..dmas5_impl).  The plan's delay
 * mode, Newton-Girard precision, cf_eps, envelope and matched filter apply;
 * its DMAS_F_CF flag does not (`variants` decides).
 *   orders_mask : bit k-1 selects order k; non-zero, no bit above the plan's
 *                 order.
 *   variants    : DMAS_V_PLAIN, DMAS_V_CF, or both.
 *   d_images    : device [V][K][M][T] float32, V = the selected variants
 *                 (plain first), K = the selected orders (ascending); each
 *                 image is the envelope (DMAS_F_ENVELOPE) or E_k (x CF).
 *   d_cf        : optional device [M][T] float32: the coherence factor.
 * The plan must have FP32 channels and order <= 5.  Each image equals that of
 * dmas_beamform with a plan of that order to FP32 rounding (not bitwise: the
 * sums differ, e.g. P_k of odd k is sum x rather than the sum of the roots'
 * k-th powers).  The first call allocates the pass's scratch (the order root
 * planes of the frame and, with the envelope, the V x K pre-envelope images)
 * and the plan keeps it; a later call that needs more grows it, which waits
 * for the device.  Same stream rule as dmas_beamform.
 * Errors: DMAS_EINVAL (NULL plan/frame/images, a plan without the pass, a bad
 * mask or variants; the reason in dmas_plan_last_error), DMAS_ENOMEM,
 * DMAS_ECUDA.
 */
dmas_status dmas_beamform_orders(dmas_plan *plan, const float *d_frame, unsigned orders_mask,
                                 int variants, float *d_images, float *d_cf, void *stream);

/*
 * Same as dmas_beamform but with HOST buffers: copies h_frame ([N][T] float32)
 * to the device, beamforms, copies the image back to h_image ([M][T] float32)
 * and synchronises `stream` before returning.  A large frame (at least 2^22
 * pixels) runs in time chunks (one per 2^21 pixels, 4 to 16) whose image
 * columns download on a second, plan-owned stream while the next chunk
 * computes; the image is bitwise the one dmas_beamform produces.  Pinned (page-locked) host memory gives the
 * fastest copies.  The device staging buffers, the copy stream and its events
 * are created on the first call and kept by the plan.  With stage profiling
 * on, the interleaved stages report as one: the whole frame under
 * "beamform".
 */
dmas_status dmas_beamform_host(dmas_plan *plan, const float *h_frame, float *h_image,
                               void *stream);

/*
 * Serving: beamform `count` frames, each with its own plan, batched.  Entries
 * that run the same kernel variant (order, delay mode, channel and
 * Newton-Girard precision, tile; for the envelope, the same taps) share one
 * launch per stage, up to 64 entries per launch, so a mixed batch costs a few
 * launches instead of three per frame; a batch of one entry is enqueued
 * exactly as dmas_beamform enqueues it.  plans/d_frames/d_images are HOST
 * arrays of `count` entries; each frame and image is a device buffer shaped as
 * for dmas_beamform.  The same plan may appear more than once (each entry gets
 * its own scratch from the workspace).  d_workspace is device memory of at
 * least dmas_batch_workspace_bytes(count, plans) bytes, 256-byte aligned, owned
 * by the caller and not used by anything else while the batch runs.  Each
 * entry's image is bitwise identical to dmas_beamform of that entry alone.
 * Errors: DMAS_EINVAL (count < 1, a NULL entry, small or misaligned
 * workspace), DMAS_ENOMEM, DMAS_ECUDA.
 */
dmas_status dmas_beamform_batch(int count, dmas_plan *const *plans,
                                const float *const *d_frames, float *const *d_images,
                                void *d_workspace, size_t workspace_bytes, void *stream);

/*
 * dmas_beamform_batch for frames held in host memory, in one call: each
 * h_frames[k] (HOST, [N][T] float32 of plans[k]; page-locked for the copy to
 * be asynchronous) is copied into the device buffer d_frames[k] on `stream`,
 * the batch is enqueued there as dmas_beamform_batch does, and `done_event`
 * (a cudaEvent_t the caller created, or NULL) is recorded after it.  The
 * caller keeps h_frames[k] unchanged until the event has fired.  Errors as for
 * dmas_beamform_batch; DMAS_EINVAL also for a NULL h_frames entry.
 */
dmas_status dmas_beamform_batch_upload(int count, dmas_plan *const *plans,
                                       const float *const *h_frames, float *const *d_frames,
                                       float *const *d_images, void *d_workspace,
                                       size_t workspace_bytes, void *stream, void *done_event);

/* Device bytes a batch of these plans needs (0 on a NULL argument). */
size_t dmas_batch_workspace_bytes(int count, dmas_plan *const *plans);

/* Device scratch bytes one dmas_beamform call of this plan uses (admission
 * control), or 0 for NULL. */
size_t dmas_plan_workspace_bytes(const dmas_plan *plan);

/* Fill *info.  Errors: DMAS_EINVAL on NULL. */
dmas_status dmas_plan_get_info(const dmas_plan *plan, dmas_plan_info *info);

/*
 * Copy the plan's delay table to host memory in the desc's direction order:
 * shift[M][N] int32 sample offsets (ROUND: llround(tau*fs); LINEAR:
 * floor(tau*fs)) and, if frac != NULL, frac[M][N] float32 interpolation weights
 * (tau*fs - floor(tau*fs) for LINEAR, 0 for ROUND).
 */
dmas_status dmas_plan_get_delays(const dmas_plan *plan, int32_t *shift, float *frac);

/* Copy the envelope taps (env_taps float32 values, h[-H..H]) to host memory. */
dmas_status dmas_plan_get_taps(const dmas_plan *plan, float *taps);

/*
 * Synchronise the plan's last stream and read the device error word that the
 * kernels set when a bounded wait expired (or, in the host-checked build, when
 * an index test failed).  Returns DMAS_OK, DMAS_ETIMEOUT, DMAS_EBOUNDS or
 * DMAS_ECUDA; clears the error word.
 *
 * Host-checked build: built beside libdmas.so as libdmas_checked.so (the same
 * sources compiled with DMAS_CHECKED), in which the beamform, every-order and
 * envelope kernels test every shared- and global-memory index they compute
 * (staged windows against their rows and shared-memory blocks, gathers
 * against their microphone's window, table copies, image rows) before the
 * access; a failing test skips the access and sets the error word, so an
 * indexing bug shows up as DMAS_EBOUNDS on a small case instead of a fault.
 */
dmas_status dmas_plan_check(dmas_plan *plan);

/* Text of the last CUDA error this plan saw ("" if none); owned by the plan. */
const char *dmas_plan_last_error(const dmas_plan *plan);

/*
 * Per-stage timing (the tracing hook of the path).  With profiling enabled a
 * dmas_beamform call records a CUDA event on its stream before and after each
 * kernel stage; nothing is skipped.  dmas_plan_stage_ms synchronises on the
 * last call's final event and writes the stage durations in milliseconds
 * (roots, beamform, envelope; 0 for a stage that did not run).
 * Errors: DMAS_EINVAL (NULL, or no profiled call yet), DMAS_ECUDA.
 */
dmas_status dmas_plan_set_profiling(dmas_plan *plan, int enable);
dmas_status dmas_plan_stage_ms(dmas_plan *plan, float *roots_ms, float *beam_ms,
                               float *env_ms);

/*
 * Scheduling of the tensor-core envelope (a serving knob; results do not
 * change).  By default its launch has one CTA per SM, each looping over its
 * share of the frame's tiles, so a big frame's envelope holds every SM until
 * it ends.  With tiles_per_cta > 0 the launch has at least
 * ceil(tiles / tiles_per_cta) CTAs, each retiring after at most that many
 * tiles, so kernels on higher-priority streams reach the SMs within a few
 * tiles' time.  0 restores the default.  Not synchronised with calls in
 * flight: set it before enqueueing work.  Errors: DMAS_EINVAL (NULL plan or a
 * negative count).
 */
dmas_status dmas_plan_set_envelope_tile_cap(dmas_plan *plan, int tiles_per_cta);

/*
 * Self-test of the kernels' bounded waits: launches one CTA that waits on a
 * shared-memory barrier no copy ever completes, with a limit of `limit_ms`
 * milliseconds (1 .. 10000).  The kernel gives up, sets its error word and
 * returns normally.  Returns DMAS_ETIMEOUT when that happened (the expected
 * result), DMAS_OK if the wait somehow completed, DMAS_EINVAL or DMAS_ECUDA.
 */
dmas_status dmas_selftest_wait_timeout(double limit_ms, void *stream);

/*
 * Beamform one frame without allocating anything.  This entry point has no
 * counterpart in the paper.  It is for callers that may allocate at set-up
 * but must not allocate while they process frames: a real-time sonar loop
 * with a fixed frame deadline, where a cudaMalloc (which can synchronise the
 * whole device and take an unbounded time) would make it miss frames, or a
 * host whose memory accounting forbids device allocations after start-up.
 *
 * It runs the same kernels as dmas_beamform with the same results, but its
 * per-call scratch (the root channels, with DMAS_F_ENVELOPE the pre-envelope
 * image, and the beamform kernel's work counter) lives in one static device
 * array of DMAS_NOALLOC_SCRATCH_BYTES that the library holds on every GPU it
 * is loaded on until the process exits.  The plan itself is created
 * beforehand with dmas_plan_create, which does allocate, once, at set-up: its
 * tables and its own scratch for dmas_beamform (dmas_plan_workspace_bytes),
 * so a plan used only through this call still holds that scratch, and the
 * static array adds its 16 MiB on each device.
 *   d_frame : device [N][T] float32;  d_image : device [M][T] float32.
 * The plan's device must be the current device.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) and keeps it for
 * the life of the process: make that first call before any stream capture,
 * and do not call cudaDeviceReset on that device afterwards (the kept address
 * would then be stale).  Every call shares the one array: calls that overlap
 * on the GPU (other streams, other threads) race and corrupt each other's
 * results, so serialise them.  Nothing from an earlier call leaks into a
 * later one: each call rewrites every byte of scratch it reads, the work
 * counter included.
 * Errors: DMAS_EINVAL (NULL argument, plan on another device, or a plan whose
 * dmas_plan_workspace_bytes exceeds DMAS_NOALLOC_SCRATCH_BYTES; the reason is
 * in dmas_plan_last_error), DMAS_ECUDA.
 */
#define DMAS_NOALLOC_SCRATCH_BYTES (16u << 20) /* 16 MiB */
dmas_status dmas_beamform_noalloc(dmas_plan *plan, const float *d_frame, float *d_image,
                                  void *stream);

/*
 * Serving runtime: frames from many sensors (each with its own plan) arrive
 * over time; a native thread batches them and launches them, so no
 * interpreter or caller thread sits between a frame's arrival and its launch.
 * This has no counterpart in the paper.
 *
 * Two lanes.  Frames whose work N*M*T is at most fast_cost take the fast lane:
 * fast_streams high-priority streams, up to max_batch frames (of any sensors)
 * per batch, one batch in flight per stream.  The others take the bulk lane:
 * one low-priority stream, one frame per batch, up to bulk_depth batches
 * queued on it at once (first in, first out, like one stream of single-frame
 * launches), overtaken on the SMs by the fast lane's kernels.  A frame is
 * admitted when its device bytes (frame, image and scratch) fit in
 * budget_bytes beside the frames in flight; a frame larger than the budget is
 * rejected (status DMAS_ENOMEM in its completion).
 *
 * The server's thread uploads each admitted frame from h_frame (page-locked
 * host memory for an asynchronous copy) into device memory it takes, with the
 * frame's image and scratch, from stream-ordered pools (cudaMallocAsync: no
 * device-wide synchronisation), runs the batch (dmas_beamform_batch_upload)
 * and copies the image to h_image when that is not NULL.  A frame submitted
 * with keep_image hands its device image to the caller in its completion
 * (free it with dmas_server_image_free); otherwise the image is freed once
 * the batch (and its copy) is done.  Times are CLOCK_MONOTONIC seconds.  The
 * caller keeps h_frame and h_image alive and unchanged until the frame's
 * completion.
 */
typedef struct dmas_server dmas_server;
typedef struct {
    int n_plans;
    dmas_plan *const *plans;   /* HOST array: one plan per sensor, not owned */
    double fast_cost;          /* N*M*T bound of the fast lane */
    int fast_streams;          /* >= 1 */
    int max_batch;             /* 1..64 frames per fast-lane batch */
    int bulk_depth;            /* >= 1 bulk-lane batches in flight */
    size_t budget_bytes;       /* device bytes of the frames in flight */
} dmas_server_desc;
typedef struct {
    uint64_t ticket;           /* from dmas_server_submit */
    int sensor;
    int status;                /* DMAS_OK, DMAS_ENOMEM (rejected) or a launch error */
    int batch_size;            /* frames in its batch */
    double t_arrival, t_admitted, t_done;  /* t_done: completion observed */
    float *d_image;            /* keep_image: the device image [M][T], else NULL */
} dmas_server_done;

/* Create a server on the current device and start its thread.  Errors:
 * DMAS_EINVAL (bad desc), DMAS_ENOMEM, DMAS_ECUDA. */
dmas_status dmas_server_create(const dmas_server_desc *desc, dmas_server **out);
/* Queue one frame of sensor `sensor` that arrived at t_arrival; *ticket
 * identifies its completion.  h_image (HOST [M][T] or NULL) receives a copy of
 * the image; keep_image != 0 hands the device image over in the completion.
 * Errors: DMAS_EINVAL, DMAS_EBUSY (server closing). */
dmas_status dmas_server_submit(dmas_server *server, int sensor, const float *h_frame,
                               float *h_image, int keep_image, double t_arrival,
                               uint64_t *ticket);
/* Free a device image a completion handed over, ordered after the work
 * already enqueued on `stream` (NULL: the legacy default stream).  It may
 * outlive the server that produced it.  NULL d_image is a no-op. */
dmas_status dmas_server_image_free(float *d_image, void *stream);
/* The next completion, waiting up to timeout_s seconds for one.  Errors:
 * DMAS_ETIMEOUT (none yet), DMAS_EINVAL. */
dmas_status dmas_server_wait(dmas_server *server, double timeout_s, dmas_server_done *out);
/* Frames queued or in flight (completions not yet taken by dmas_server_wait
 * are not counted). */
int dmas_server_pending(dmas_server *server);
/* Stop accepting frames, finish the ones queued and in flight, stop the
 * thread and free everything; completions not yet taken are dropped.  NULL
 * is a no-op. */
dmas_status dmas_server_destroy(dmas_server *server);

/* Static text for a status code. */
const char *dmas_status_string(dmas_status status);

/* Library version as major*10000 + minor*100 + patch. */
int dmas_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DMAS_H */
