/*
 * xcorr.h -- C ABI of the GB300 X-stage: cross-multiply and integrate for an
 * FX radio correlator.
 *
 * What the library computes (Sec. 1 and Sec. 2.1 of the paper: the X-stage
 * forms, for every frequency channel and time sample, the outer product of
 * the spectra of all inputs and integrates the products over time; Sec. 2.2.3,
 * Eq. 1: all N_i (N_i + 1) / 2 input pairs, autocorrelations included):
 *
 *     V[c][i][j] = sum_t x[t][c][i] * conj(x[t][c][j]),   0 <= j <= i < N_i
 *
 * with N_i = 2 * n_stations inputs, input i = 2 * station + pol (the paper's
 * N_i counts two inputs per antenna, Sec. 2.2.3).  The integration is the
 * exact SUM over the samples given since the last reset; the paper's GPU
 * averages (Sec. 2.4, Sec. 4), and the caller divides by the sample count
 * returned with each dump.
 *
 * Input layout (Sec. 2.3 and Fig. 3: per time sample, every channel of every
 * input), sample order [time][channel][station][pol], one element per
 * complex sample:
 *   XCORR_IN_CI4   uint8: high nibble = real, low nibble = imaginary, each
 *                  4-bit two's complement in [-8, 7] (Sec. 2.3: four bits
 *                  per component; the nibble order is this library's
 *                  reading, the paper does not fix it).
 *   XCORR_IN_CI8   int8 pair (re, im), the unpacked 8-bit form of Sec. 2.4.
 *   XCORR_IN_CF32  float pair (re, im), spectra from a GPU F-stage (Sec. 1).
 *                  Each input's samples are quantised per 384-sample window
 *                  against the window's largest magnitude (23 bits) and split
 *                  into three integer digits; the six leading digit products
 *                  are summed exactly per window and scaled into a float
 *                  accumulator.  The error is about 1e-7 of
 *                  sqrt(|V_ii V_jj|) per entry (at most 1e-6).
 *                  Edge values, all handled without flushing:
 *                  - subnormal samples, and whole windows of them, are
 *                    quantised on a grid of 2^-149 or finer, which holds
 *                    every float exactly, so any finite input keeps the
 *                    bound above (there is no lower magnitude limit);
 *                  - results are float: an entry whose exact value lies below
 *                    the normal float range (2^-126) comes out as a float
 *                    subnormal or zero; one whose partial sums pass the
 *                    float range (about 3.4e38) comes out non-finite (+-inf,
 *                    or NaN where partial sums of both signs overflow);
 *                  - a NaN or +-inf sample makes every entry that pairs its
 *                    input with any input (its own autocorrelation
 *                    included) NaN, re and im, in that channel, for the rest
 *                    of the integration and in every dump that holds it; all
 *                    other entries are unaffected.  Where the exact sum has
 *                    a non-finite term, so does this result (NaN where the
 *                    FP64 sum has an inf or a NaN).
 *
 * Output layout: the packed lower triangle per channel, pair index
 * p(i, j) = i (i + 1) / 2 + j for i >= j, (re, im) interleaved:
 * [channel][pair][2].  Element type: int32 for CI4 / CI8, float for CF32;
 * with XCORR_DUMP_ADD_WIDE the caller's buffer is int64 / double instead.
 * V[c][j][i] = conj(V[c][i][j]) is not stored.
 *
 * Threading and ordering: a plan may be used by one host thread at a time.
 * execute and dump are stream-ordered and return without waiting for the GPU
 * unless stated; plan_create and destroy synchronise the device.
 *
 * Errors: every call returns an xcorr_status and never aborts the process;
 * xcorr_last_error() gives a message for the calling thread's last failure.
 * Kernel-side failures (a bounded wait that ran out) are recorded in a device
 * status word; xcorr_sync reports them, and every later call on the plan
 * returns XCORR_ERR_DEVICE until xcorr_destroy.
 */
#ifndef XCORR_H
#define XCORR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    XCORR_OK = 0,
    XCORR_ERR_INVALID_ARG = 1,  /* a size, pointer, alignment or flag is invalid          */
    XCORR_ERR_UNSUPPORTED = 2,  /* valid request this build or device cannot serve       */
    XCORR_ERR_OOM = 3,          /* device allocation failed                              */
    XCORR_ERR_OVERFLOW = 4,     /* the integration would exceed the exact int32 range   */
    XCORR_ERR_CUDA = 5,         /* a CUDA runtime call failed (message has the detail)  */
    XCORR_ERR_DEVICE = 6,       /* a kernel reported a failure (bounded wait timed out) */
    XCORR_ERR_BUDGET = 7        /* the plan's device memory exceeds hbm_budget_bytes    */
} xcorr_status;

typedef enum { XCORR_IN_CI4 = 0, XCORR_IN_CI8 = 1, XCORR_IN_CF32 = 2 } xcorr_in_fmt;

typedef enum {
    XCORR_ENGINE_AUTO = 0,      /* the faster engine as measured on GB300: CUDA-core at
                                   most 16 channels with fewer than 16 inputs (CI4) or at
                                   most 64 inputs (CI8), the tensor cores otherwise       */
    XCORR_ENGINE_TENSOR = 1,    /* tcgen05 tensor-core X kernel                          */
    XCORR_ENGINE_CUDA_CORE = 2  /* plain CUDA-core (dp4a) X kernel, integer formats only */
} xcorr_engine;

typedef struct {
    int n_stations;          /* >= 1; N_i = 2 * n_stations inputs                       */
    int n_pols;              /* must be 2 (dual polarisation, Sec. 2.2.3)               */
    int n_channels;          /* >= 1                                                    */
    int max_time_per_exec;   /* >= 1; largest n_time one xcorr_execute may pass         */
    xcorr_in_fmt fmt;
    xcorr_engine engine;
    size_t hbm_budget_bytes; /* 0 = no limit; else plan_create fails with BUDGET above it */
} xcorr_config;

typedef struct xcorr_plan_s *xcorr_plan;

/* Launch shape of the tensor-core path (xcorr_plan_set_tuning, xcorr_autotune). */
typedef struct {
    int stage_variant;  /* shared-memory ring, 0 .. 10: planes path 0 = 3 x 64 KB, 1 (and 3 .. 10)
                           = 4 x 48 KB, 2 = 6 x 32 KB stages; fused path see `unfused`         */
    int groups;         /* channel groups whose unpack overlaps the X kernel; 0 = automatic (<= 8) */
    int x_streams;      /* 1 or 2 streams the groups' X launches alternate over                 */
    int unfused;        /* 4-bit input: 0 = unpack on chip inside the X kernel where possible
                           (N_i % 16 == 0, 16-byte aligned input); stage_variant then picks
                           raw / decoded rings of 128 x (2 + 2), 96 x (4 + 2), 64 x (6 + 3)
                           samples with 8 decoder warps, or 96 x (4 + 2) with 12 (both
                           operands decoded into shared memory); 4 .. 6: the A operand
                           decoded into tensor memory, raw / decoded rings of
                           128 x (2 + 2), 96 x (3 + 2), 64 x (4 + 4) samples (4 is the
                           default of a 4-bit plan); 7 .. 9: pairs of SMs (a thread-block
                           cluster of 2, one cta_group::2 MMA) sharing a column tile,
                           rings of 96 x (2 + 3), 128 x (2 + 2), 128 x (2 + 3) samples;
                           10: the tensor-memory-A kernel's small-problem layout,
                           128 x (2 + 2): for N_i <= 64, 128 / N_i channels side by
                           side in one 128-row tile; and when a launch has fewer tiles
                           than SMs, each tile's stages split over several CTAs whose
                           sums are added atomically into the (cleared) output;
                           1 = always through E4M3 planes in HBM                            */
} xcorr_tuning;

/* Opaque to the caller except through these fields (xcorr_plan_query). */
typedef struct {
    int n_inputs;             /* N_i = 2 * n_stations                                    */
    int n_channels;
    int64_t n_pairs;          /* N_i (N_i + 1) / 2                                       */
    int engine;               /* the engine actually selected (never AUTO)               */
    int64_t samples_integrated; /* samples accumulated since the last reset              */
    int64_t max_integration;  /* most samples one integration may hold exactly in int32 */
    size_t device_bytes;      /* device memory the plan owns                             */
    size_t output_bytes;      /* bytes of one dump in the plan's own element type        */
    int kernels_per_execute;  /* kernel launches of one full-size execute (unpack + X)   */
    xcorr_tuning tuning;      /* current launch shape (groups resolved)                  */
} xcorr_plan_info;

/*
 * Create a plan.  Validates cfg, allocates the device accumulator and any
 * staging buffers on the current device (the plan owns them), and selects the
 * kernels.  *out receives the plan, or NULL on failure.
 * Engines: TENSOR uses the tcgen05 kernels for every format (4-bit as E4M3,
 * int8 as BF16, float as three BF16 pieces); CUDA_CORE takes CI4 / CI8; AUTO
 * takes CUDA_CORE for at most 16 channels with fewer than 16 inputs (CI4) or at
 * most 64 inputs (CI8), where its single launch was measured faster than the
 * tensor path's unpack + X, and TENSOR otherwise.  A 4-bit tensor plan starts on
 * launch shape 10 (the small-problem layout) when N_i <= 64 and either
 * max_time_per_exec >= 1024 or n_channels >= 256, else on shape 4.
 * max_integration (xcorr_plan_query) is 16,777,215 samples for CI4, 65,535
 * for CI8 (exact int32) and 16,777,216 for CF32 (longer sums: dump with
 * XCORR_DUMP_ADD_WIDE into double).
 * Errors: INVALID_ARG (bad sizes, n_pols != 2, NULL pointers), UNSUPPORTED
 * (no GB300-class device, or CF32 with the CUDA-core engine), OVERFLOW
 * (max_time_per_exec beyond max_integration), BUDGET, OOM, CUDA.
 */
xcorr_status xcorr_plan_create(xcorr_plan *out, const xcorr_config *cfg);

/*
 * Correlate n_time samples and add them to the running integration
 * (Sec. 2.1: cross multiplication and integration per channel and sample).
 * d_in: caller-owned DEVICE memory, [n_time][n_channels][n_stations][2]
 * samples in the plan's format (CI4 and CI8 at any alignment, CF32 4-byte
 * aligned; 16-byte alignment and N_i a multiple of 16 take the vectorised
 * paths), read-only; it must stay valid until the stream passes this call.
 * 1 <= n_time <= max_time_per_exec.
 * stream: a cudaStream_t (NULL = the legacy default stream).
 * Errors: INVALID_ARG (also a CF32 pointer that is not 4-byte aligned),
 * OVERFLOW (samples since reset + n_time would exceed
 * max_integration; nothing is launched), DEVICE, CUDA.
 */
xcorr_status xcorr_execute(xcorr_plan plan, const void *d_in, int n_time, void *stream);

/* Flags for xcorr_dump. */
#define XCORR_DUMP_RESET 1u     /* start a new integration after this dump               */
#define XCORR_DUMP_ADD_WIDE 2u  /* out is int64 (CI4/CI8) or double (CF32) device memory,
                                   and the integration is ADDED to it (the cross-dump
                                   accumulation of Sec. 2.4 / Sec. 4, kept exact)        */

/*
 * Write the current integration to out in the output layout above.
 * out_on_device != 0: out is device memory (required with ADD_WIDE);
 * otherwise out is host memory (pinned for a truly asynchronous copy).
 * *n_samples (may be NULL) receives the samples in this integration, the
 * divisor of the paper's average.  The copy is stream-ordered: read out only
 * after synchronising the stream.  Errors: INVALID_ARG, DEVICE, CUDA.
 */
xcorr_status xcorr_dump(xcorr_plan plan, void *out, int out_on_device, unsigned flags,
                        void *stream, int64_t *n_samples);

/*
 * Resume an integration (checkpoint / restart; Sec. 2.4: the dumps are the
 * correlator's durable product).  src holds a dump taken without
 * XCORR_DUMP_RESET in the layout xcorr_dump writes -- int32 [C][P][2] for
 * CI4 / CI8, float [C][P][2] for CF32, C * P * 8 bytes, host memory or
 * (src_on_device != 0) device memory -- and n_samples, the samples it
 * integrates (the count that dump reported).  The plan takes it as its
 * running sums: later executes add to it, later dumps include it, and the
 * integration's sample count continues from n_samples.  The copy is
 * stream-ordered; src may be reused once the stream has passed it.  The plan
 * must hold no integration (new, or dumped with XCORR_DUMP_RESET).
 * Errors: INVALID_ARG (NULL src, n_samples < 0, the plan holds an
 * integration), OVERFLOW (n_samples > max_integration), DEVICE, CUDA.
 */
xcorr_status xcorr_accum_load(xcorr_plan plan, const void *src, int src_on_device, int64_t n_samples,
                              void *stream);

/*
 * xcorr_execute followed by xcorr_dump with the same flags, in one call.
 * When this execute is the whole integration (the plan was reset, flags
 * hold XCORR_DUMP_RESET and not ADD_WIDE, and out is device memory) the X
 * kernel writes the visibilities straight into out and the plan's own
 * accumulator is not touched; otherwise it is exactly the two calls.
 * Sec. 2.1 / Sec. 2.4: the GPU integrates and hands the matrix back.
 * Errors: those of xcorr_execute and xcorr_dump.
 */
xcorr_status xcorr_execute_dump(xcorr_plan plan, const void *d_in, int n_time, void *out,
                                int out_on_device, unsigned flags, void *stream,
                                int64_t *n_samples);

/*
 * One whole integration from host memory to host memory, with the copies
 * overlapped with the X-stage: the channels are cut into n_groups groups (0 =
 * the library's choice: at most 8, each copy row at least 64 KB, since copy
 * engines move narrower 2-D rows at half rate); each group's input columns go up (a 2-D
 * copy of its channels of every sample), are correlated, and its triangle
 * comes back while later groups are still being copied or correlated.  The
 * result equals copying the input to the device, xcorr_execute_dump with
 * XCORR_DUMP_RESET, and copying the output back.  h_in: n_time samples in the
 * input layout; h_out: [C][P][2] as xcorr_dump writes it.  Both should be
 * pinned (cudaHostAlloc / cudaHostRegister), or the copies do not overlap.  The
 * plan must hold no integration (nothing executed since the last reset) and
 * still holds none afterwards.  Input that the fused 4-bit kernel cannot take
 * (other formats, the CUDA-core engine, unaligned sizes) runs as one piece:
 * the copy up, the X-stage and the copy down, in order.  The first call
 * allocates a device copy of one input (max_time_per_exec samples), kept
 * until xcorr_destroy.  Stream-ordered on `stream`.
 * Errors: INVALID_ARG, OVERFLOW, OOM, CUDA, DEVICE.
 */
xcorr_status xcorr_execute_dump_host(xcorr_plan plan, const void *h_in, int n_time, void *h_out, int n_groups,
                                     void *stream);

/* Wait for the stream and report any kernel-side failure (DEVICE). */
xcorr_status xcorr_sync(xcorr_plan plan, void *stream);

/*
 * Check the failure path of the kernels' bounded waits.  This enqueues one
 * kernel whose wait can never complete: an mbarrier that nothing arrives at.
 * The wait gives up after the library's wait limit (2 s) and records a
 * timeout in the plan's status word, exactly as a stalled X-stage kernel
 * would.  The next xcorr_sync then returns XCORR_ERR_DEVICE, and the plan
 * refuses every later call until xcorr_destroy.  No GPU fault is involved,
 * and other plans on the device keep working.  Errors: INVALID_ARG, CUDA,
 * DEVICE.
 */
xcorr_status xcorr_watchdog_selftest(xcorr_plan plan, void *stream);

/*
 * Fix the tensor path's launch shape (results do not depend on it).
 * Errors: INVALID_ARG (stage_variant not in [0, 10], groups not in [0, 8],
 * x_streams not 1 or 2), DEVICE.
 */
xcorr_status xcorr_plan_set_tuning(xcorr_plan plan, const xcorr_tuning *tuning);

/*
 * Autotuner: time every launch shape of the tensor path on this input (three
 * runs each, the first as warm-up), keep the fastest on the plan and return it
 * in *best (and its time in ms in *best_ms; either may be NULL).  Discards the
 * plan's current integration.  Synchronises the stream.  A CUDA-core plan has
 * nothing to tune and returns at once.  Errors: INVALID_ARG, CUDA, DEVICE.
 */
xcorr_status xcorr_autotune(xcorr_plan plan, const void *d_in, int n_time, void *stream,
                            xcorr_tuning *best, float *best_ms);

/*
 * The autotuner with a cache of its results (the paper has no counterpart; the
 * paper's deployment retunes nothing, but a correlator serving many subarray
 * sizes should not time every shape at every start).  If the process's tuning
 * cache holds a shape for this plan's problem -- the device's name and SM
 * count, the input format, N_i, the channel count and n_time -- the shape is
 * applied without timing and *from_cache is 1; otherwise xcorr_autotune runs
 * and its winner is recorded in the cache (*from_cache 0).  Either way the
 * plan's current integration is discarded, as by xcorr_autotune.  best,
 * best_ms (the recorded time) and from_cache may be NULL.
 * Errors: as xcorr_autotune.
 */
xcorr_status xcorr_autotune_cached(xcorr_plan plan, const void *d_in, int n_time, void *stream,
                                   xcorr_tuning *best, float *best_ms, int *from_cache);

/*
 * The process's tuning cache, in files.  save writes every entry, one JSON
 * object per line with the fields scope ("plan" or "batch"), device, sms, fmt,
 * n_inputs, n_channels, n_time, stage_variant, groups, x_streams, unfused,
 * us (the recorded time, microseconds) and shape_table (the revision of this
 * library's table of launch shapes, which gives stage_variant its meaning);
 * the file is replaced whole (written to path.tmp, then renamed).  load
 * merges a file's entries into the cache (an entry for the same problem is
 * replaced); a line without every field, with a value out of range, or from
 * another shape-table revision is skipped and counted in *n_skipped.  clear
 * empties the cache.  n_loaded, n_skipped and n_saved may be NULL.
 * Errors: INVALID_ARG (NULL path, a file that cannot be opened or written).
 */
xcorr_status xcorr_tuning_cache_load(const char *path, int *n_loaded, int *n_skipped);
xcorr_status xcorr_tuning_cache_save(const char *path, int *n_saved);
xcorr_status xcorr_tuning_cache_clear(void);

/* Describe the plan.  Errors: INVALID_ARG. */
xcorr_status xcorr_plan_query(xcorr_plan plan, xcorr_plan_info *info);

/*
 * Kernel timing for benchmarks (no counterpart in the paper).  With
 * capacity > 0 every later execute records CUDA events on the streams its
 * kernels run on: at its start, after its last unpack kernel, and before and
 * after every launch of the X kernel (the tensor path may split the channels
 * into groups, each with its own launch; the CUDA-core engine has no unpack).
 * The last `capacity` executes are kept; capacity 0 turns timing off.
 * Errors: INVALID_ARG, CUDA.
 */
xcorr_status xcorr_profile_enable(xcorr_plan plan, int capacity);

/*
 * Wait for the recorded events and write, oldest first, two durations in ms
 * per timed execute: ms[2k] from the start of the execute to the end of its
 * last unpack kernel, ms[2k + 1] the summed durations of its X-kernel launches.
 * `capacity` is the number of executes ms has room for; *count receives how
 * many were written.  Errors: INVALID_ARG, CUDA.
 */
xcorr_status xcorr_profile_read(xcorr_plan plan, float *ms, int capacity, int *count);

/*
 * Measure a dense arithmetic rate of the current device in tera-operations
 * per second (two operations per multiply-add), for stating fractions of
 * peak; no counterpart in the paper.  kind 0: tcgen05 E4M3 MMA (the tensor
 * X kernel's instruction), 1: tcgen05 BF16 MMA, 2: the int8 tensor path of
 * sm_103a (warp-level mma.sync s8; tcgen05 has no int8 kind there), 3: CUDA-
 * core dp4a.  Runs for tens of milliseconds and synchronises the device.
 * Errors: INVALID_ARG, CUDA, DEVICE.
 */
xcorr_status xcorr_measure_peak(int kind, double *tops);

/*
 * One-shot 4-bit correlation that allocates no memory (the paper has no
 * counterpart; this serves callers that cannot allocate when they correlate,
 * such as a real-time capture loop in which cudaMalloc would synchronise the
 * device and stall the streams draining the network, or code whose device
 * memory belongs to another framework's fixed pool).
 *
 * Computes the same packed-triangle visibilities as a tensor-engine plan:
 * d_in is CI4 device memory [n_time][n_channels][n_stations][2] (any
 * alignment), d_out receives int32 [n_channels][P][2] (device memory, written,
 * not added to).  d_status, if not NULL, is a device int that receives the
 * kernels' status word (0 = success).  Both buffers are the caller's.
 * d_status is the only way to learn that a kernel's bounded wait ran out
 * (the call has already returned XCORR_OK by then, and d_out is then only
 * partly written): callers should pass it and check it after the stream
 * passes the call.
 *
 * The staging planes live in a fixed 64 MiB array that every GPU loading the
 * library holds until the process exits; a call needs
 * 2 * n_channels * n_time * round_up(2 * n_stations, 16) bytes of it and is
 * refused with INVALID_ARG beyond 64 MiB - 256 bytes.  The array's device
 * address is looked up on every call whose stream is not being captured, so
 * it follows a cudaDeviceReset or a change of CUDA context; a call on a
 * capturing stream reuses the address last seen for that device and context,
 * so the first call on a device (and after a reset or in a new context) must
 * come before any stream capture.  Every call uses the same array and leaves its
 * contents behind, so calls whose work overlaps on the GPU (different
 * streams, or different host threads) race and must be serialised by the
 * caller.  The call returns without waiting for the GPU.
 * Errors: INVALID_ARG, OVERFLOW, UNSUPPORTED, CUDA.
 */
xcorr_status xcorr_correlate_ci4_noalloc(const void *d_in, int n_time, int n_channels,
                                         int n_stations, void *d_out, int *d_status,
                                         void *stream);

/*
 * Batches: many independent 4-bit correlations of uneven size (each its own
 * station count, channel count and integration length; Sec. 2.1: each
 * sub-band is an independent X-stage) in one persistent tensor-core launch
 * over the union of their tile pairs, longest first, so small subarrays fill
 * the tail of the large ones.  When every subarray has a multiple of 16
 * inputs and at most 37,248 samples, the launch is the fused 4-bit kernel
 * (A operand in tensor memory) reading d_ins directly (16-byte aligned);
 * otherwise each execute first unpacks every subarray into staging planes the
 * batch owns.  Subarray s correlates exactly cfgs[s].max_time_per_exec
 * (<= 130,944) samples per execute from d_ins[s] ([t][c][s][2] CI4, device)
 * into d_outs[s] (int32 [C][P][2], device, written, not added to).  The
 * caller owns the buffers.
 */
typedef struct xcorr_batch_s *xcorr_batch;

/* Errors: INVALID_ARG, UNSUPPORTED (a non-CI4 subarray, a device that is not
 * sm_103a, more than 130,944 samples), BUDGET (sum of planes over the
 * smallest nonzero hbm_budget_bytes), OOM, CUDA. */
xcorr_status xcorr_batch_create(xcorr_batch *out, const xcorr_config *cfgs, int n);

/* The launch shape: 0, 1, 2 for the planes path's rings (as in xcorr_tuning),
 * 3, 4, 5 for the fused kernel's (as xcorr_tuning's 4, 5, 6; 3 is the default
 * of a batch that qualifies).  Errors: INVALID_ARG, UNSUPPORTED (a fused shape
 * for a batch that does not qualify), OOM (the planes of a planes shape). */
xcorr_status xcorr_batch_set_variant(xcorr_batch batch, int stage_variant);

/* A shape per subarray (fused batches only): variants[s] is a 4-bit plan
 * shape, xcorr_tuning.stage_variant 0 .. 10 with unfused = 0.  Subarrays whose
 * shape is one of the tensor-memory-A kernel's (4, 5, 6) form a class with its
 * own item list and one shared launch; a subarray with any other shape (the
 * CTA-pair kernel 7-9, the small-problem layout 10, the shared-memory kernel
 * 0-3) runs as its own launch.  All of these run side by side on internal
 * streams forked from (and joined back to) the caller's stream, inside a
 * captured graph too.  xcorr_batch_set_variant(3 + k) sets every subarray to
 * plan shape 4 + k.  get reads the current shapes (the batch-wide shape 0-2,
 * repeated, for the planes path).  Errors: INVALID_ARG, UNSUPPORTED (a batch
 * the fused kernel does not take). */
xcorr_status xcorr_batch_set_subarray_variants(xcorr_batch batch, const int *variants);
xcorr_status xcorr_batch_get_subarray_variants(xcorr_batch batch, int *variants);

/* Autotuner of a batch (the paper has no counterpart): per subarray, the
 * fused plan shape (0 .. 10) that runs it fastest on its own, timed with these
 * buffers (three runs each, the first as warm-up; d_outs are overwritten), or
 * taken without timing from the process's tuning cache (scope "batch", see
 * xcorr_tuning_cache_save), where every new result is recorded.  The shapes
 * are applied as by xcorr_batch_set_subarray_variants and written to
 * variants (n entries; may be NULL).  A batch on the planes path has one
 * shape and nothing to tune.  Synchronises the stream.  Errors: INVALID_ARG
 * (NULL or unaligned buffers), CUDA, DEVICE. */
xcorr_status xcorr_batch_autotune(xcorr_batch batch, const void *const *d_ins, void *const *d_outs, void *stream,
                                  int *variants);

/* One batch execute on the stream.  Errors: INVALID_ARG (a NULL buffer, or an
 * input the fused kernel cannot read: not 16-byte aligned), CUDA. */
xcorr_status xcorr_batch_execute(xcorr_batch batch, const void *const *d_ins, void *const *d_outs,
                                 void *stream);

/* Capture one batch execute with these buffers into a CUDA graph (the
 * buffers must stay valid while the graph is replayed).  Errors: INVALID_ARG,
 * CUDA. */
xcorr_status xcorr_batch_capture(xcorr_batch batch, const void *const *d_ins, void *const *d_outs,
                                 void *stream);

/* Launch the captured graph on the stream.  Errors: INVALID_ARG, CUDA. */
xcorr_status xcorr_batch_replay(xcorr_batch batch, void *stream);

/* Wait for the stream and report kernel-side failures (DEVICE). */
xcorr_status xcorr_batch_sync(xcorr_batch batch, void *stream);

/* Synchronise the device and free the batch.  NULL is a no-op. */
xcorr_status xcorr_batch_destroy(xcorr_batch batch);

/*
 * Streaming: the receive side of the paper's X-stage server (Sec. 2.3,
 * Sec. 2.4, Fig. 3, Fig. 4) on one GPU.  F-engine packets land in pinned host
 * chunks, go to the device, and a scatter kernel places each payload by its
 * (sequence number, F-engine id) into a device ring of n_blocks blocks of
 * block_samples samples ([t][c][i] CI4, the layout xcorr_execute reads); that
 * placement is the corner turn the paper's capture and unpack threads do.
 * Packets may arrive in any order.  While the oldest block is incomplete,
 * packets of later blocks are held in their own ring blocks (the paper's
 * stack); when their number reaches stack_threshold, or a packet arrives for
 * a block past the ring, the oldest block is closed: its missing packets are
 * recorded lost and zero-filled, and it is correlated into the current dump.
 * A complete oldest block closes at once.  Every blocks_per_dump blocks (the
 * integration K = blocks_per_dump * block_samples) the dump is copied to a
 * pinned host buffer, asynchronously.
 *
 * Packet format (Sec. 2.3, Fig. 3): XCORR_PACKET_HEADER_BYTES of header -- a
 * 64-bit little-endian sequence number, a 32-bit little-endian F-engine id and
 * 4 unused bytes -- then n_time_per_packet spectra one after another, each
 * n_chan_per_packet channels x n_inputs_per_packet inputs of CI4 bytes
 * ([t][channel][input]).  F-engine f sends inputs [f N_a, (f + 1) N_a); its
 * sequence number counts its own packets: seq = time_block * n_groups +
 * channel_group with n_groups = n_channels / n_chan_per_packet, time_block
 * covering samples [time_block N_t, (time_block + 1) N_t).  Block b holds
 * samples [b * block_samples, (b + 1) * block_samples).
 */
#define XCORR_PACKET_HEADER_BYTES 16

typedef struct {
    int n_time_per_packet;     /* N_t, >= 1                                                  */
    int n_chan_per_packet;     /* divides the plan's n_channels                              */
    int n_inputs_per_packet;   /* N_a: a multiple of 16 that divides n_inputs                */
    int block_samples;         /* a multiple of N_t, <= the plan's max_time_per_exec         */
    int n_blocks;              /* blocks in the device ring, >= 2 (the paper's rings hold 4) */
    int blocks_per_dump;       /* >= 1; K = blocks_per_dump * block_samples <= the plan's
                                  exact integration bound                                    */
    int64_t stack_threshold;   /* >= 1: held packets of later blocks that close the oldest   */
    int64_t chunk_packets;     /* packets per pinned landing chunk, >= 1                     */
    int n_chunks;              /* landing chunks, >= 2                                       */
    int n_host_dumps;          /* pinned host dump buffers, >= 1                             */
} xcorr_stream_config;

/* Packet accounting, cumulative. */
typedef struct {
    int64_t packets;        /* headers seen                                         */
    int64_t placed;         /* distinct packets placed in the ring                  */
    int64_t duplicates;     /* a (seq, F-engine) already placed in an open block    */
    int64_t late;           /* for a block already closed                           */
    int64_t bad;            /* F-engine id out of range                             */
    int64_t lost;           /* never received by the time their block closed        */
    int64_t blocks_closed;
} xcorr_packet_counters;

/*
 * Host-side packet tracking, the decision logic of the stream without the
 * GPU (usable from a capture thread, and testable on any host).
 * xcorr_tracker_feed reads n headers (packet k at packets + k * stride) and
 * writes codes[k] = (ring slot << 40) | packet index within the block, or -1
 * when the packet is dropped (duplicate, late, bad).  The packet index of
 * (time block tb in its block, channel group g, F-engine f) is
 * (tb * n_groups + g) * n_fengines + f.  Each block event (an OPEN when a
 * block takes a ring slot, a CLOSE when the oldest block is closed) is
 * reported with the packet position in this call at which it takes effect.
 * Processing stops early when max_events are reported; *n_done gives the
 * packets consumed.  Errors: INVALID_ARG.
 */
typedef struct xcorr_tracker_s *xcorr_tracker;

#define XCORR_EVENT_OPEN 1
#define XCORR_EVENT_CLOSE 2

typedef struct {
    int kind;          /* XCORR_EVENT_OPEN or XCORR_EVENT_CLOSE                           */
    int slot;          /* ring slot (block % n_blocks)                                    */
    int64_t block;     /* block index                                                     */
    int64_t position;  /* packets of this call before the event                           */
    int64_t received;  /* CLOSE: distinct packets placed in the block                     */
    int64_t lost;      /* CLOSE: packets of the block never received                      */
} xcorr_block_event;

xcorr_status xcorr_tracker_create(xcorr_tracker *out, const xcorr_stream_config *cfg, int n_inputs,
                                  int n_channels);
xcorr_status xcorr_tracker_feed(xcorr_tracker tr, const void *packets, int64_t stride, int64_t n,
                                int64_t *codes, xcorr_block_event *events, int max_events,
                                int *n_events, int64_t *n_done);
/* Close every open block (end of stream).  Same event rules. */
xcorr_status xcorr_tracker_finish(xcorr_tracker tr, xcorr_block_event *events, int max_events,
                                  int *n_events);
xcorr_status xcorr_tracker_counters(xcorr_tracker tr, xcorr_packet_counters *out);
xcorr_status xcorr_tracker_destroy(xcorr_tracker tr);

/*
 * Cut CI4 samples [n_time][n_channels][n_inputs] (host, n_time a multiple of
 * N_t) into packets in the order an F-engine array sends them: for each time
 * block, each channel group, each F-engine.  Time block tb of the samples is
 * time block first_time_block + tb of the stream.  Writes
 * (n_time / N_t) * n_groups * n_fengines packets of 16 + N_t * N_ch * N_a
 * bytes to `packets` (host).  Errors: INVALID_ARG (sizes, capacity).
 */
xcorr_status xcorr_packetize(const void *samples, int n_time, int n_channels, int n_inputs,
                             const xcorr_stream_config *cfg, int64_t first_time_block,
                             void *packets, int64_t capacity_packets, int64_t *n_packets);

/*
 * Add seq_delta to the sequence number of n packets (packet k's header at
 * packets + k * stride, host memory): replays the same payloads as later time
 * blocks, the way an F-engine emulator keeps a link busy without rewriting
 * payloads.  Errors: INVALID_ARG.
 */
xcorr_status xcorr_packets_advance(void *packets, int64_t stride, int64_t n, int64_t seq_delta);

typedef struct xcorr_stream_s *xcorr_stream;

typedef struct {
    int64_t index;         /* dump number: block / blocks_per_dump                          */
    int64_t first_seq;     /* sequence number of channel group 0 of the dump's first
                              sample (Sec. 2.3: time stamps follow from the sequence numbers):
                              index * blocks_per_dump * block_samples / N_t * n_groups      */
    int64_t n_samples;     /* samples integrated (blocks correlated x block_samples)        */
    int64_t lost_packets;  /* zero-filled packets in this dump's blocks                     */
    double latency_ms;     /* host time from closing the dump's last block to its copy
                              being in host memory                                          */
    const void *data;      /* pinned host copy, int32 [C][P][2], valid until n_host_dumps
                              later dumps with data are issued; NULL when n_samples == 0
                              or when that has already happened                            */
} xcorr_dump_record;

/*
 * Create a stream over a CI4 plan (which it drives; do not execute the plan
 * meanwhile).  The stream's device memory (ring, landing chunks, two dump
 * buffers) plus the plan's must fit the plan's hbm_budget_bytes when that is
 * nonzero.  Errors: INVALID_ARG, UNSUPPORTED (not CI4), BUDGET, OOM, CUDA.
 */
xcorr_status xcorr_stream_create(xcorr_stream *out, xcorr_plan plan, const xcorr_stream_config *cfg);

/* The next landing chunk to fill with up to *capacity_packets packets (pinned
 * host memory owned by the stream); waits until its previous contents reached
 * the device.  Errors: INVALID_ARG, CUDA. */
xcorr_status xcorr_stream_acquire(xcorr_stream s, void **chunk, int64_t *capacity_packets);

/* Hand over the first n_packets of the acquired chunk: headers are tracked on
 * the host, the chunk goes to the device and is scattered; closed blocks are
 * correlated and finished dumps copied out, all asynchronously.
 * Errors: INVALID_ARG, CUDA, DEVICE. */
xcorr_status xcorr_stream_commit(xcorr_stream s, int64_t n_packets);

/* End of stream: close every open block and issue the last (partial) dump. */
xcorr_status xcorr_stream_flush(xcorr_stream s);

/* Dumps issued so far, and the packet counters. */
xcorr_status xcorr_stream_counters(xcorr_stream s, xcorr_packet_counters *counters,
                                   int64_t *dumps_issued);

/* Wait up to timeout_ms for the k-th dump issued (0-based) to reach host
 * memory.  Errors: INVALID_ARG (k not issued yet), CUDA (timeout: the
 * stream's copies did not finish), DEVICE. */
xcorr_status xcorr_stream_wait_dump(xcorr_stream s, int64_t k, int timeout_ms, xcorr_dump_record *rec);

/* Synchronise the stream's work and free it (not the plan).  NULL is a no-op. */
xcorr_status xcorr_stream_destroy(xcorr_stream s);

/*
 * Baseline-dependent integration (Sec. 6: short baselines rotate their fringes
 * slowly and can be integrated longer without decorrelation; per-baseline
 * integration lengths lower the output data rate).  The triangle of input
 * pairs is cut into 128 x 128 tile pairs: input blocks I >= J of 128 inputs,
 * tile pair t = I (I + 1) / 2 + J, nb = ceil(N_i / 128) blocks, nb (nb + 1) / 2
 * tile pairs.  Tile pair t integrates over cadence[t] >= 1 base integrations.
 *
 * A base integration is whatever was executed on the plan since its last
 * reset.  xcorr_bdi_step then, in one pass over the triangle on the stream:
 *  - adds the plan's integration into the running sums of every tile pair;
 *  - resets the plan;
 *  - emits the tile pairs due at this step, those with
 *    (step + 1) % cadence[t] == 0, where steps count from 0.
 *
 * Output layout: out receives the due tile pairs as dense blocks, int32
 * [n_due][C][128][128][2]. Row r, column q of block k is the pair
 * (128 I_k + r, 128 J_k + q). It is zero where that pair is not stored: past
 * N_i, or above the diagonal. The due tile pairs' running sums restart from
 * zero.
 *
 * Host-side outputs: due[] (capacity nb (nb + 1) / 2) receives the emitted
 * tile-pair indices in increasing order, samples[] their integration lengths,
 * and *n_due their count. out may be device memory (out_on_device = 1) or host
 * memory.
 *
 * Integer (CI4, CI8) plans only.  The running sums live in a device buffer of
 * the plan's output size.
 * Errors: INVALID_ARG, UNSUPPORTED (float input), OVERFLOW (a tile pair would
 * integrate past the plan's exact bound; nothing changes), OOM, CUDA, DEVICE.
 */
typedef struct xcorr_bdi_s *xcorr_bdi;

xcorr_status xcorr_bdi_create(xcorr_bdi *out, xcorr_plan plan, const int *cadence, int n_tile_pairs);
xcorr_status xcorr_bdi_step(xcorr_bdi bdi, void *out, int out_on_device, void *stream, int *n_due, int *due,
                            int64_t *samples);
/* Synchronise the device and free the running sums.  NULL is a no-op. */
xcorr_status xcorr_bdi_destroy(xcorr_bdi bdi);

/* Synchronise the device, free the plan's memory and the plan.  NULL is a no-op. */
xcorr_status xcorr_destroy(xcorr_plan plan);

/* Message for the calling thread's last failed call ("" if none).  Owned by the library. */
const char *xcorr_last_error(void);

/*
 * Map a station pair and polarisation product to the packed triangle
 * (recovers the view of Eq. 4, baselines times four polarisation products, from
 * the input-pair triangle).  V(a, p; b, q) = x_{a,p} conj(x_{b,q}) for
 * stations a >= b, pols p, q in {0, 1}.  *idx receives p(i, j) of the stored
 * pair and *conj is 1 when the requested product is the conjugate of the
 * stored one (only for a == b, p < q).  Errors: INVALID_ARG.
 */
xcorr_status xcorr_baseline_index(int n_stations, int a, int b, int p, int q, int64_t *idx,
                                  int *conj);

#ifdef __cplusplus
}
#endif
#endif /* XCORR_H */
