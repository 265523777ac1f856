/*
 * fdas.h -- C ABI of the GB300 (sm_103a) FDAS frequency-domain convolution library.
 *
 * The library computes the filter-output plane of the Fourier-domain acceleration
 * search (Sec. 3): one long complex single-precision Fourier-domain array x[0..N)
 * is convolved with a bank of M complex FIR templates h_z[0..K) (Eq. 1,
 * y_z[i] = sum_{k<K} x[i-k] h_z[k], i = 0..N-1, x[j] = 0 for j < 0), and the
 * spectral power P[z][i] = |y_z[i]|^2 is stored (Sec. 4.3: power, no square root).
 * The convolution is evaluated by overlap-save (Algorithm 2, Sec. 3.2.2) with one
 * forward FFT per input segment shared by all templates (Table 1 and its text).
 *
 * Conventions
 *   - complex64 = two IEEE float32 (re, im), interleaved, 8 bytes per value;
 *   - the power plane is float32, row-major [M][n]: row z holds template z in the
 *     order the templates were given to fdas_plan_create;
 *   - "stream" is a cudaStream_t passed as void* (NULL = the legacy default stream);
 *   - device pointers belong to the caller and must stay valid until the work
 *     queued on the stream has finished; the plan owns only its own device state;
 *   - every entry point returns 0 (FDAS_OK) or a negative FDAS_ERR_* code and never
 *     throws; fdas_last_error() gives a thread-local message for the last failure.
 *   - entry points that enqueue GPU work are asynchronous unless stated otherwise.
 */
#ifndef FDAS_H
#define FDAS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FDAS_OK                 0
#define FDAS_ERR_INVALID_ARG   (-1)   /* null pointer, size out of range, misaligned pointer */
#define FDAS_ERR_OOM           (-2)   /* a device or pinned-host allocation failed */
#define FDAS_ERR_CUDA          (-3)   /* a CUDA runtime/driver call failed (see fdas_last_error) */
#define FDAS_ERR_TIMEOUT       (-4)   /* a bounded wait (host deadline or in-kernel spin) ran out */
#define FDAS_ERR_BUSY          (-5)   /* server: no free slot or budget right now */
#define FDAS_ERR_REJECTED      (-6)   /* server: request can never fit the memory budget */
#define FDAS_ERR_UNSUPPORTED   (-7)   /* option value not built into this library */

/* Arithmetic forms of the segment FFTs. */
#define FDAS_PREC_FP32          0     /* FP32 CUDA-core FFTs (default) */
#define FDAS_PREC_TC_FP16       1     /* the inverse FFT's first radix-16 pass as a tensor-core
                                         DFT-GEMM: fp16 data, fp16 hi/lo-split DFT matrix, FP32
                                         accumulation; the other passes FP32; needs seg_len 2048 */
#define FDAS_PREC_TC_DFT2       2     /* the whole inverse FFT as two tensor-core DFT-GEMMs
                                         (2048 = 32 x 64: fp16 operands, FP32 accumulation, the
                                         product with H_z fused into the first operand, the twiddle
                                         and |y|^2 on the CUDA cores); the forward FFT FP32 with a
                                         per-segment power-of-two range scale; needs seg_len 2048 */

typedef struct fdas_plan_s *fdas_plan;

/* Plan options; a zero-initialised struct (or NULL) selects the defaults. */
typedef struct {
    int seg_len;      /* L, the overlap-save FFT length: 1024, 2048 or 4096 (0 = 2048) */
    int tpl_per_cta;  /* G, templates per thread block: 1..M; 0 = chosen per call from the number
                         of segments (all M for long arrays, fewer per block for short ones so
                         that the launch still fills the GPU; the tensor-core form uses all M) */
    int precision;    /* FDAS_PREC_* (0 = FP32) */
    int autotune;     /* 1: time every (L in {1024, 2048, 4096}) x (G chosen per call, 5, 17, 85)
                         with the persistent batch kernel on a seeded proxy of the batches the
                         plan will serve (16 arrays, lengths log-uniform in [tune_n_min, n_max])
                         and keep the fastest (seg_len is then ignored; a non-zero tpl_per_cta
                         stays fixed); 2: the same, with the two-stage tensor-core form
                         (FDAS_PREC_TC_DFT2, L = 2048, its 2e-3 tolerance) as one more candidate.
                         Results are cached per process by (device, M, K, lengths, mode, G) */
    int group_support;/* 1: group the templates by the length of their nonzero support, each
                         group with its own overlap-save frame and step and its templates stored
                         shifted to their first nonzero tap (fewer inverse FFTs when supports
                         differ); one launch per group.  FP32 form, without autotuning; used by
                         fdas_convolve, fdas_convolve_host and fdas_convolve_candidates (the
                         batched and served forms return FDAS_ERR_UNSUPPORTED for such a plan) */
    int64_t tune_n_min;  /* autotuner: shortest array of the proxy batch (0 = n_max / 16) */
} fdas_opts;

/* Read-only description of a plan. */
typedef struct {
    int64_t n_max;        /* largest array length accepted */
    int     n_templates;  /* M */
    int     tpl_len;      /* K as given */
    int     frame_len;    /* K used internally: K padded with up to 3 trailing zero taps so that
                             frame_len - 1 is a multiple of 4 (the convolution is unchanged) */
    int     seg_len;      /* L */
    int     seg_step;     /* S: valid outputs per segment, a multiple of 4, <= L - frame_len + 1 */
    int     tpl_per_cta;  /* G (0: chosen per call) */
    int     precision;    /* FDAS_PREC_* */
    int     device;       /* CUDA device ordinal the plan lives on */
    int64_t device_bytes; /* device memory owned by the plan */
    int     tuned;        /* 1 if the autotuner chose seg_len, tpl_per_cta (and precision) */
    float   tune_ms[12];  /* autotuner: ms per proxy batch, [L in 1024, 2048, 4096][G in per call, 5, 17, 85] (0 = not run) */
    float   tune_ms_tc;   /* autotuner (mode 2): ms per proxy batch of the two-stage tensor-core form */
    int     batch_blocks; /* blocks of the persistent batch kernel (resident blocks per SM x SMs) */
    int     groups;       /* template groups = kernel launches per plane (1 unless group_support) */
} fdas_plan_desc;

/*
 * fdas_plan_create -- build a plan for arrays of up to n_max points.
 *
 *   templates_c64_host : host pointer, complex64 [n_templates][tpl_len], row-major.
 *                        Copied during the call; the caller keeps ownership.
 *   n_templates        : M >= 1.   tpl_len : K, 1 <= K <= L - 4.
 *   opts               : NULL or options (see fdas_opts).
 *
 * Synchronous.  Allocates on the current CUDA device and runs the plan-time kernels:
 * the FP64 twiddle tables and the FP64 transform of every zero-padded template,
 * H_z = FFT_L(h_z) / L (Algorithm 2, "Fourier transform of coefficient array"; its
 * cost is left out of Table 1 because N >> K), stored as FP32 in the order the
 * segment kernel consumes it.
 * Errors: INVALID_ARG (bad sizes or options), UNSUPPORTED, OOM, CUDA.
 */
int fdas_plan_create(fdas_plan *out, int64_t n_max, const void *templates_c64_host,
                     int n_templates, int tpl_len, const fdas_opts *opts);

/* Fill *desc with the plan's parameters.  Errors: INVALID_ARG. */
int fdas_plan_describe(fdas_plan p, fdas_plan_desc *desc);

/* Templates per thread block that fdas_convolve uses for an array of n points (the plan's
 * fixed G, or the per-call choice when the plan was created with tpl_per_cta = 0; a grouped
 * plan applies the same rule to each template group and its segment count).
 * Returns G >= 1, or a negative error code (INVALID_ARG for a null plan or n outside
 * [1, n_max]).  Host only; no CUDA call. */
int fdas_plan_tpl_per_cta(fdas_plan p, int64_t n);

/*
 * fdas_convolve -- power plane of one array (the hot path).
 *
 *   in_c64_dev    : device pointer, complex64 [n], 16-byte aligned.
 *   n             : 1 <= n <= n_max.
 *   out_power_dev : device pointer, float32 [M][n] row-major, 4-byte aligned; every
 *                   element is written.  Must not overlap the input.
 *
 * Enqueues one kernel launch on `stream` (one per template group for a plan created
 * with group_support) and returns without waiting.  Per segment
 * of L points (step S, preceded by K-1 zeros for the first, zero-filled past n):
 * one forward FFT, then for each template the element-wise product, the inverse
 * FFT, the discard of the first K-1 points and the power (Algorithm 2, Sec. 4.3).
 * Errors: INVALID_ARG, CUDA (launch failure).  Asynchronous faults surface on the
 * stream; bounded in-kernel waits that run out are reported by fdas_plan_status.
 */
int fdas_convolve(fdas_plan p, const void *in_c64_dev, int64_t n, float *out_power_dev,
                  void *stream);

/*
 * fdas_convolve_direct -- the same plane by the time-domain form: Eq. (1) evaluated term
 * by term (8NK operations per template, Table 1 "TD naive") on the CUDA cores, then |y|^2.
 * For the filter-length comparison with overlap-save (Sec. 6, latency against filter
 * length); arguments, layout and errors as fdas_convolve.  Asynchronous.
 */
int fdas_convolve_direct(fdas_plan p, const void *in_c64_dev, int64_t n, float *out_power_dev,
                         void *stream);

/* One threshold crossing of the power plane. */
typedef struct {
    int32_t tpl;     /* template (row) index */
    float   power;   /* P[tpl][bin], bit-identical to the plane fdas_convolve writes */
    int64_t bin;     /* output index i, 0 <= i < n */
} fdas_candidate;

/*
 * fdas_convolve_candidates -- the candidates of one array instead of its plane.
 *
 * The FT-convolution module sends the power plane on to candidate detection (Sec. 3);
 * this entry point fuses the first step of that, the threshold, into the store epilogue
 * of the segment kernel: every (tpl, bin) with P[tpl][bin] > threshold is appended to
 * cand_dev, and the plane itself is never written to memory.
 *
 *   in_c64_dev : device complex64 [n], 16-byte aligned;  1 <= n <= n_max.
 *   cand_dev   : device array of max_cand fdas_candidate (max_cand >= 0).
 *   count_dev  : device pointer to one unsigned 64-bit counter; the library clears it on
 *                `stream` before the launch; afterwards it holds the number of crossings
 *                found, which may exceed max_cand (then only max_cand were stored).
 * The order of the stored candidates is unspecified.  Asynchronous.  FP32 and two-stage
 * tensor-core (FDAS_PREC_TC_DFT2) plans; for the latter the crossings and their powers are those
 * of the plane that form writes, bit for bit.
 * Errors: INVALID_ARG, UNSUPPORTED (an FDAS_PREC_TC_FP16 plan), CUDA.
 */
int fdas_convolve_candidates(fdas_plan p, const void *in_c64_dev, int64_t n, float threshold,
                             fdas_candidate *cand_dev, int64_t max_cand,
                             unsigned long long *count_dev, void *stream);

/*
 * fdas_convolve_host -- the same computation from and to host memory.
 *
 *   in_c64_host    : host complex64 [n];  out_power_host : host float32 [M][n].
 *   Pinned (page-locked) buffers give full copy bandwidth; pageable ones work.
 *
 * Synchronous: copies the input to plan-owned device staging memory (allocated on
 * the first call, sized for n_max), runs the segment kernel in chunks and copies
 * each finished chunk of the plane back while the next one is computed (a grouped
 * plan: all launches, then one copy), and returns once out_power_host is complete.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
int fdas_convolve_host(fdas_plan p, const void *in_c64_host, int64_t n, float *out_power_host,
                       void *stream);

/*
 * fdas_convolve_batch -- power planes of `count` arrays of uneven lengths in one
 * persistent launch (the dedispersion trials of a beam share the templates).
 *
 *   ins[i]  : device pointer, complex64 [ns[i]], 16-byte aligned;  1 <= ns[i] <= n_max.
 *   outs[i] : device pointer, float32 [M][ns[i]] row-major, 4-byte aligned.
 *   The three arrays of pointers/lengths are host memory, read during the call.
 *
 * Enqueues, per group of up to 120 arrays, one replay of the plan's CUDA graph
 * [reset the work counter -> persistent kernel with one block per resident slot].  FP32
 * plans: the kernel's blocks take work items (array, template group, segment) from the
 * counter.  FDAS_PREC_TC_DFT2 plans: one block per SM takes an equal share of the launch's
 * (array, segment pair, template pair) units.  Each template's arithmetic is that of
 * fdas_convolve (whatever the grouping), so results equal those of fdas_convolve on each
 * array bit for bit.  Asynchronous.  Calls on one plan are serialised by the library on the
 * host; their kernels run in stream order and must not overlap in time: do not
 * issue batches of one plan on two streams that run concurrently.
 * Errors: INVALID_ARG (any entry invalid: nothing is enqueued), UNSUPPORTED (a plan
 * created with group_support, or an FDAS_PREC_TC_FP16 plan, for which this form is not
 * built; nothing is enqueued), CUDA.
 */
int fdas_convolve_batch(fdas_plan p, int count, const void *const *ins, const int64_t *ns,
                        float *const *outs, void *stream);

/*
 * fdas_convolve_batch_noalloc -- fdas_convolve_batch without any allocation in the call.
 *
 * The paper has no counterpart: this entry point exists for callers that cannot
 * allocate GPU memory while they run, e.g. a real-time pipeline that must meet a
 * per-trial deadline (cudaMalloc can take milliseconds and cudaFree synchronises the
 * device), or a process whose device memory is owned up front by another allocator.
 * It computes the same planes as fdas_convolve_batch (same arguments, same kernel,
 * same work items) but allocates nothing: no cudaMalloc/cudaFree, no CUDA graph, no
 * heap memory; the persistent kernel's work counters live in a fixed array of 64
 * ints that the library places in every GPU's memory for the life of the process.
 *
 *   count <= 7680 (64 launches of up to 120 arrays); larger batches are rejected with
 *   FDAS_ERR_INVALID_ARG and a message naming the limit.  Other arguments as for
 *   fdas_convolve_batch.
 *
 * The first call on a device looks up the counter array's device address (once per
 * device, with the plan's device current); make that first call before any stream
 * capture.  Each call clears the counters it uses on `stream` before its launches.
 * All calls in the process share the one array: calls whose work overlaps on the GPU
 * (different streams, different plans, or different threads without ordering) race
 * on it and must be serialised by the caller.  Asynchronous.
 * A device reset (cudaDeviceReset) destroys the counter array with the context; the
 * address looked up before it is not looked up again, so after a reset this entry point
 * must not be called again in the same process.
 * Errors: INVALID_ARG, UNSUPPORTED (as fdas_convolve_batch), CUDA.
 */
int fdas_convolve_batch_noalloc(fdas_plan p, int count, const void *const *ins, const int64_t *ns,
                                float *const *outs, void *stream);

/*
 * fdas_plan_status -- wait for `stream`, then read and clear the plan's device
 * status word.  Returns FDAS_OK, FDAS_ERR_TIMEOUT if an in-kernel bounded wait ran
 * out since the last call, or FDAS_ERR_CUDA if the stream reports an error.
 */
int fdas_plan_status(fdas_plan p, void *stream);

/*
 * Failure-detection self-test: enqueues on `stream` one block whose bounded mbarrier wait
 * runs out after limit_ms (0 < limit_ms <= 1000) because it waits for a copy that is never
 * issued -- the path a segment kernel takes when a TMA load never lands.  The block sets the
 * plan's status word and exits; no copy is in flight and the context stays usable.  The next
 * fdas_plan_status returns FDAS_ERR_TIMEOUT (and clears the word).  Errors: INVALID_ARG, CUDA.
 */
int fdas_selftest_wait_timeout(fdas_plan p, double limit_ms, void *stream);

/*
 * Full-length frequency-domain FIR (Eq. 2; the "naive FDFIR" of Sec. 3.2.1 and Table 1), the
 * alternative the paper weighs overlap-save against: y_z = IFFT_P(FFT_P(x) . FFT_P(h_z)) with
 * P the smallest power of two >= n_max + tpl_len - 1 (at least 2^21, at most 2^23), then
 * |y_z[i]|^2 for i < n -- the same plane as fdas_convolve (Eq. 1), computed with P-point
 * transforms of the whole array (four-step, P = 2048 x P/2048) instead of segments.
 *
 * fdas_fdfir_create: synchronous; copies the M x K complex64 templates (host, row-major) and
 *   stores their P-point spectra on the current device (M x P x 8 bytes: 5.7 GB for 85
 *   templates at P = 2^23).  Errors: INVALID_ARG (null pointers, sizes < 1, n_max + tpl_len - 1
 *   > 2^23), OOM, CUDA.
 * fdas_fdfir_length: *P = the transform length.
 * fdas_fdfir_convolve: enqueues on `stream` (2 + 2M kernel launches) the plane out[z][i]
 *   (float32, [M][n] row-major, device) of in[0, n) (complex64, device, 8-byte aligned);
 *   1 <= n <= n_max; in and out must not overlap.  Calls on one plan share its scratch and
 *   must not overlap on the GPU.  Errors: INVALID_ARG, CUDA.
 * fdas_fdfir_destroy: frees the plan (the caller has synchronised its streams).
 */
typedef struct fdas_fdfir_s *fdas_fdfir;
int fdas_fdfir_create(fdas_fdfir *out, int64_t n_max, const void *templates_c64_host, int n_templates, int tpl_len);
int fdas_fdfir_length(fdas_fdfir f, int64_t *P);
int fdas_fdfir_convolve(fdas_fdfir f, const void *in_c64_dev, int64_t n, float *out_power_dev, void *stream);
int fdas_fdfir_destroy(fdas_fdfir f);

/* ------------------------------------------------------------------------------------
 * Harmonic summing of a power plane (the module that receives the plane, Sec. 3; the
 * paper names it without defining it, read here as the incoherent harmonic sum).
 *
 * Rows are ordered by drift: row y holds drift z = y - c, c = (n_templates - 1) / 2 (the
 * order of the bank z = -c .. c); column bin0 holds frequency bin 0 (templates centred in a
 * frame of F taps delay the plane by (F - 1) / 2 bins: bin0 = 210 for 421-tap frames).  The
 * k-th harmonic of a signal at bin r with drift z lies at bin k r with drift k z, so for the
 * fundamental (r, z), r >= 1,
 *     S_h(r, z) = sum_{k=1..h} P[c + k z][bin0 + k r]     (FP32, added for k = 1, 2, ..)
 * for h = 1, 2, 4, .., max_harm, defined where |h z| <= c and bin0 + h r <= n - 1.
 * ---------------------------------------------------------------------------------- */
typedef struct {
    int32_t tpl;       /* row of the fundamental, c + z */
    float   power;     /* S_h */
    int64_t bin;       /* column of the fundamental, bin0 + r */
    int32_t nharm;     /* h */
    int32_t reserved;  /* 0 */
} fdas_harmonic_candidate;

/*
 * fdas_harmonic_sum -- every defined S_h(r, z) > thresholds[log2 h] is appended to cand_dev.
 *
 *   plane_dev   : device float32 [n_templates][n], row-major, 4-byte aligned (the plane
 *                 fdas_convolve writes); n_templates odd; n >= 1; 0 <= bin0 < n.
 *   max_harm    : 1, 2, 4, 8, 16 or 32.
 *   thresholds  : host float [log2(max_harm) + 1], one per level h = 1, 2, .., max_harm.
 *   cand_dev    : device array of max_cand records (8-byte aligned; may be null if
 *                 max_cand = 0).
 *   count_dev   : device unsigned 64-bit counter (8-byte aligned), cleared on `stream`
 *                 before the launch; afterwards the number of crossings, which may exceed
 *                 max_cand (then only max_cand were stored).
 * Runs on the current device; the order of the records is unspecified.  Asynchronous: one
 * memset, then one kernel launch on `stream` per run of rows with the same number
 * min(max_harm, c / |z|) of harmonics inside the drift range (at most 2 max_harm - 1
 * launches; a single launch for rows of more than 2^31 - 2^16 bins; none when no fundamental
 * fits).  Errors: INVALID_ARG, CUDA.
 */
int fdas_harmonic_sum(const float *plane_dev, int n_templates, int64_t n, int64_t bin0, int max_harm,
                      const float *thresholds, fdas_harmonic_candidate *cand_dev, int64_t max_cand,
                      unsigned long long *count_dev, void *stream);

/* ------------------------------------------------------------------------------------
 * Served form: continuous batching over one plan.
 *
 * Requests (device input arrays) are admitted in arrival order as soon as the memory
 * for their planes (4*M*n bytes, rounded up to 256) is free in a pool reserved once at
 * creation; admitted requests are packed into batches of up to max_batch arrays and
 * launched on whichever of the `lanes` streams is idle, so a request that arrives while
 * others run on the GPU starts as soon as a lane and memory free up, and batches on
 * different lanes overlap on the device.  The plan (templates, transforms, kernels)
 * stays resident; the plan must outlive the server.  A request's plane stays in the
 * pool until fdas_server_release.  Each request's plane equals fdas_convolve's for the
 * same input (same kernel, same work items).
 * ---------------------------------------------------------------------------------- */
typedef struct fdas_server_s *fdas_server;

typedef struct {
    int64_t budget_bytes;  /* device memory for output planes, reserved at creation (> 0) */
    int     lanes;         /* concurrent batch streams, 1..16 (0 = 2) */
    int     max_batch;     /* arrays per launch, 1..120 (0 = 32) */
} fdas_server_opts;

typedef struct {
    int64_t submitted, completed, rejected;
    int64_t queued;            /* waiting for plane memory */
    int64_t in_flight;         /* admitted and not yet released */
    int64_t bytes_in_use, peak_bytes_in_use;
    int64_t admission_waits;   /* requests that could not be admitted when submitted */
    int64_t launches;          /* batch launches */
    double  p50_ms, p99_ms, mean_ms, max_ms;   /* latency: submit -> plane complete on the GPU */
    double  arrays_per_s;      /* completed / (last completion - first submission) */
} fdas_server_report;

/* Create a server (starts its scheduler thread; reserves budget_bytes on the plan's
 * device).  FP32 and FDAS_PREC_TC_DFT2 plans.  Errors: INVALID_ARG, UNSUPPORTED (a grouped
 * plan, or an FDAS_PREC_TC_FP16 plan), OOM, CUDA. */
int fdas_server_create(fdas_server *out, fdas_plan plan, const fdas_server_opts *opts);

/* Queue one request.  in_c64_dev: device complex64 [n], 16-byte aligned, valid until
 * the request completes; 1 <= n <= n_max.  Non-blocking.  *ticket identifies it.
 * Errors: INVALID_ARG, REJECTED (its plane alone exceeds the budget). */
int fdas_server_submit(fdas_server s, const void *in_c64_dev, int64_t n, int64_t *ticket);

/* Wait until the request's plane is complete (timeout_ms < 0: no limit); *plane_dev
 * (optional) receives its device address, float32 [M][n].  Errors: INVALID_ARG
 * (unknown ticket), TIMEOUT, CUDA (the launch failed). */
int fdas_server_wait(fdas_server s, int64_t ticket, int64_t timeout_ms, float **plane_dev);

/* Return a completed request's plane memory to the pool.  Errors: INVALID_ARG, BUSY
 * (still queued or running). */
int fdas_server_release(fdas_server s, int64_t ticket);

/* Counters and latency percentiles since creation or the last reset. */
int fdas_server_stats(fdas_server s, fdas_server_report *report);
int fdas_server_reset_stats(fdas_server s);

/* Stop the scheduler, let launched batches finish, free the pool and the lanes;
 * planes not yet launched are dropped. */
int fdas_server_destroy(fdas_server s);

/* Free the plan.  The caller must have synchronised every stream that used it. */
int fdas_destroy(fdas_plan p);

/* Static description of an FDAS_* code. */
const char *fdas_strerror(int code);

/* Thread-local message of the most recent failure on the calling thread ("" if none). */
const char *fdas_last_error(void);

/* Library version string. */
const char *fdas_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FDAS_H */
