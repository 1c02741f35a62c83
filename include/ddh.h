/*
 * libddh — Dynamic DH-MBIR per-frame EM step on one GB300 (sm_103a).
 *
 * C ABI: plain pointers and sizes only.  Every compute step runs in the library's own CUDA
 * kernels; there is no CPU path.  All calls are asynchronous on the CUDA stream given to
 * ddh_init() unless stated otherwise; errors found by the device (non-finite frame, a bounded
 * wait that expired) are latched in a device status word and returned by the next call that
 * synchronises (ddh_sync, ddh_phase/ddh_reflectance to host memory, ddh_strehl).  A call
 * that works on a state makes the state's device current for its duration and restores the
 * calling thread's current device before it returns.
 *
 * Method: Sheikh, Pellizzari, Kisner, Buzzard, Bouman, "Dynamic DH-MBIR for Phase-Error
 * Estimation from Streaming Digital-Holography Data" (arXiv:2305.03284).  Per frame (Fig. 1):
 * Normalize (Eq. 4), RemoveTipTilt (Sec. 4), r-init (Eq. 3), N_k EM iterations (Sec. 3) on the
 * isoplanatic model y = D_a D(exp(j phi)) F g + w (Eq. 1, Sec. 2).
 *
 * Layouts: an N x N image is row-major (index = row * N + col, row = y, col = x).  Frames are
 * interleaved complex64 (re, im float pairs).  The aperture D_a is the disc of diameter
 * `aperture_diam` px centred on ((N-1)/2, (N-1)/2).
 */
#ifndef DDH_H_
#define DDH_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes (negative) ------------------------------------------------------------ */
#define DDH_OK 0
#define DDH_EINVAL (-1)      /* bad argument (NULL, unsupported N, misaligned pointer, ...) */
#define DDH_ENOMEM (-2)      /* device allocation failed */
#define DDH_ECUDA (-3)       /* a CUDA runtime call failed (see ddh_last_cuda_error) */
#define DDH_ETIMEOUT (-4)    /* a bounded device wait expired; that frame left the state as is */
#define DDH_ENONFINITE (-5)  /* frame had a non-finite entry or zero variance; state unchanged */
#define DDH_EBUDGET (-6)     /* admission refused: the memory budget would be exceeded */

/* ---- parameters (Fig. 1 arguments lambda, alpha, N_k; Sec. 5.B values) -------------------- */
typedef struct ddh_params {
  int n;                /* grid side N: 32, 64, 128, 256 (cluster kernel) or 512 (L2-staged kernels) */
  float aperture_diam;  /* pupil diameter in px, 0 < d <= N */
  float lambda;         /* Eq. 3 weight of the back-projection term (paper: 0.45) */
  float alpha;          /* Eq. 3 scale of |A^H y|^2 (paper: 0.025) */
  int n_k;              /* EM iterations per frame, 1..1024 (paper: 1; the static DH-MBIR mode
                           uses one bootstrap period, 200 in the paper) */
  float noise_var;      /* sigma^2 of the noise after Normalize (> 0) */
  float prior_p;        /* q-GGMRF shape p, 1 <= p < 2 */
  float prior_q;        /* q-GGMRF shape q; must be 2 (finite surrogate weight at 0) */
  float prior_T;        /* q-GGMRF threshold T > 0 */
  float prior_sigma;    /* q-GGMRF scale sigma_r > 0 */
  float r_floor;        /* lower bound on the reflectance (> 0) */
  int tilt_mode;        /* 1: RemoveTipTilt each frame; 0: skip it */
  int phase_block;      /* 1: per-pixel phase; 2 or 4: phase constant on aligned G x G tiles,
                           phi_B = angle(sum over the tile of a y~ conj(F mu)) */
  float phase_prior;    /* p(phi) of Eq. 2 on the tiles (the paper defers its form): precision
                           1/sigma_phi^2 of a Gaussian MRF on the wrapped differences of
                           8-neighbour tiles; the tile-phase M-step then minimises
                           -(2/sigma^2) sum_t |v_t| cos(phi_t - angle v_t) + prior by
                           `phase_sweeps` majorised 4-colour ICD sweeps from the tile angles.
                           0 (default): flat prior.  > 0 needs phase_block 2 or 4, n_k = 1 and
                           a pupil of at most 128 x 128 tiles (any grid and exec_path, e.g.
                           512^2 with a 256 px pupil in 2 x 2 tiles); in batches and the
                           service the streams that use it share one post-step launch */
  int phase_sweeps;     /* ICD sweeps of that M-step, 1..16 (0 counts as the default, 2) */
  int noise_update;     /* 1: sigma^2 (noise_var above is then its starting value) is
                           re-estimated once per frame, after the frame's last EM iteration, by
                           its EM M-step (1/|P|) sum_pupil |y~ - e^{j phi} F mu|^2 + mean(C);
                           floored at 1e-6.  Any grid and exec_path, also in batches and the
                           service; no adjoint.  0 (default): sigma^2 fixed */
  int exec_path;        /* which kernels run this stream's steps (same method, same readings;
                           results agree within FP32 rounding, not bit for bit):
                           DDH_PATH_DEFAULT (0): the cluster kernel for N <= 256, the L2-staged
                           kernels for N = 512; DDH_PATH_CLUSTER (1): one thread-block cluster
                           per stream holds the whole frame in shared memory (N <= 256; lowest
                           latency for one stream); DDH_PATH_STAGED (2): a sequence of batched
                           kernels over per-stream global scratch that stays in L2 (N = 128,
                           256 or 512; uses every SM when many streams step together, so the
                           higher throughput for large batches).  Fixed for the state's
                           lifetime: a stream steps the same way alone and in any batch.  The
                           staged path has no trace output, host-buffer in-place steps or
                           adjoint (DDH_EINVAL); the tile-phase prior and the sigma^2 M-step run
                           on both paths */
} ddh_params;
#define DDH_PATH_DEFAULT 0
#define DDH_PATH_CLUSTER 1
#define DDH_PATH_STAGED 2

typedef struct ddh_state ddh_state; /* opaque; owned by the library */

/* Fill `p` with the defaults for grid `n`, pupil `aperture_diam` and a linear SNR over the
 * pupil: lambda 0.45, alpha 0.025 (Sec. 5.B), n_k 1, noise_var 1/(1 + f SNR) with f the
 * pupil fill fraction, prior p 1.1, q 2, T 1, sigma_r 0.1, r_floor 1e-10, tilt_mode 1,
 * phase_block 1, phase_prior 0, phase_sweeps 2, noise_update 0, exec_path DDH_PATH_DEFAULT. */
int ddh_default_params(ddh_params *p, int n, float aperture_diam, float snr);

/* Static DH-MBIR (Sec. 3: EM iterated on one frame, the reflectance reset to a back-projected
 * estimate every `reset_every` iterations) is the frame step with lambda = 1, alpha = 1,
 * n_k = reset_every and tilt_mode = 0: each ddh_step on the same frame then resets
 * r = |A_phi^H y~|^2 with the current phase (Eq. 3 with lambda = alpha = 1) and runs one
 * bootstrap period of EM iterations; phi carries over.  This fills `p` with those values on
 * top of ddh_default_params. */
int ddh_static_params(ddh_params *p, int n, float aperture_diam, float snr, int reset_every);

/* The parameter set under which the one-iteration-per-frame loop tracks frozen-flow
 * turbulence on a bar-chart object at the paper's simulation parameters (Sec. 5.A: D/r0 10,
 * 0.42 px/frame in x and y, SNR 10 dB), reaching a Strehl ratio of 0.8 within 150 frames as
 * Sec. 5.C reports: ddh_default_params with the phase on 2 x 2 tiles under the Gaussian MRF
 * tile prior (phase_block 2, phase_prior 10), q-GGMRF scale sigma_r 0.03 and alpha 0.0125
 * (Eq. 3; the best value of a grid search over [0, 0.1], the paper's own range, on that
 * workload; the paper's 0.025 was found on its data). */
int ddh_tracking_params(ddh_params *p, int n, float aperture_diam, float snr);

/* Validate `p`, allocate the device state (r = 0, phi = 0, n = 0: Fig. 1 first line) and bind
 * it to `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).  The library owns
 * the state until ddh_free().  Returns DDH_OK or DDH_EINVAL / DDH_ENOMEM / DDH_ECUDA. */
int ddh_init(ddh_state **out, const ddh_params *p, void *cuda_stream);

/* One DDH-MBIR time step (Fig. 1 loop body) on frame `y_c64_dev`: device pointer to N*N
 * interleaved complex64, 16-byte aligned, caller-owned; it must stay valid until the step has
 * run in stream order.  Enqueues one kernel launch and returns; a non-finite frame is
 * reported later (DDH_ENONFINITE) and leaves r and phi unchanged. */
int ddh_step(ddh_state *s, const void *y_c64_dev);

/* Same step, also writing the frame's intermediates into `trace_dev` (N <= 256) (device, float32,
 * ddh_trace_floats(N) entries): b = A^H y (complex, N*N), mu (complex, N*N), z = F mu
 * (complex, N*N), r-init (N*N), s = E|g|^2 (N*N), then 8 scalars (mean re, mean im, scale,
 * t_x, t_y, 0, 0, 0).  Complex fields are interleaved; all images row-major. */
int ddh_step_trace(ddh_state *s, const void *y_c64_dev, float *trace_dev);
size_t ddh_trace_floats(int n);

/* One step from HOST memory: the frame from `y_c64_host`, phi (N*N float32) to `phi_host_out`,
 * and waits for completion.  Pinned, mapped buffers are read and written in place by the step
 * kernel (the conditions of ddh_step_host_async); otherwise the frame is copied into a device
 * staging buffer owned by the state and phi copied out after the step. */
int ddh_step_host(ddh_state *s, const void *y_c64_host, float *phi_host_out);

/* Pipelined form of ddh_step_host: enqueues the frame's step and returns at once with
 * `*ticket` = this frame's sequence number on the state.  When both host buffers are pinned and
 * mapped into the device's address space (cudaHostAlloc / torch pin_memory), N <= 256 and
 * neither post-step M-step (phase_prior, noise_update) is on, the step kernel reads the frame
 * and writes phi over the CPU-GPU link itself: one launch per frame, no staging copies (the
 * same results bit for bit).  Otherwise the frame is copied in on a library copy stream into
 * one of two device staging slots, so that frame n+1's copy overlaps frame n's step, and phi is
 * copied out after the step.  Both buffers stay untouched until ddh_host_wait(s, ticket) or
 * ddh_sync(s) returns (pageable memory makes the staged copies synchronous).  Errors latched
 * by the step (non-finite frame, timeout) surface at ddh_sync.  Steps of one state must not be
 * enqueued from several threads at once.  The paper has no counterpart (it describes a frame
 * loop, not its host interface). */
int ddh_step_host_async(ddh_state *s, const void *y_c64_host, float *phi_host_out, int64_t *ticket);
/* Block until frame `ticket` of ddh_step_host_async has its phi in host memory (DDH_EINVAL
 * for a ticket not issued on s). */
int ddh_host_wait(ddh_state *s, int64_t ticket);

/* WriteData (Fig. 1): stream-ordered copy of phi_n / r_n (N*N float32) into `out`, which may
 * be device or host memory (host copies synchronise the stream and report latched errors). */
int ddh_phase(const ddh_state *s, float *out);
int ddh_reflectance(const ddh_state *s, float *out);

/* Overwrite the state (r, phi: N*N float32, device or host pointers) and the frame count;
 * used to resume from a checkpoint and by teacher-forced comparisons. */
int ddh_set_state(ddh_state *s, const float *r, const float *phi, int64_t frame_index);
int64_t ddh_frame_index(const ddh_state *s);
/* The sigma^2 the next frame's E-step will use: the running estimate when noise_update is on
 * (synchronises the state's stream), else noise_var.  ddh_init, ddh_set_params and
 * ddh_set_state (re)start the estimate at noise_var; checkpoints carry it. */
int ddh_noise_estimate(ddh_state *s, float *out);
/* Replace the state's parameters by `p` (validated; same N, else DDH_EINVAL), keeping r, phi,
 * the frame count and the device buffers.  Host-side only: calls enqueued afterwards use the
 * new values (each launch takes its parameters by value), work already enqueued keeps the old
 * ones.  A ddh_batch created before the call keeps the old values (create it again).  Used to
 * reuse one state across calls whose prior or noise parameters differ (training through the
 * unrolled adjoint updates them every iteration); not thread-safe against other calls on s. */
int ddh_set_params(ddh_state *s, const ddh_params *p);
/* The cudaStream_t the state's work is ordered on (the one given to ddh_init, or the service's
 * stream for a state admitted by ddh_service_admit); NULL if s is NULL. */
void *ddh_state_stream(const ddh_state *s);

/* Peak Strehl ratio of the current phase estimate against `phi_true_dev` (N*N float32, device):
 * max |F^H(a exp(j(phi_true - phi)))|^2 / max |F^H a|^2 (Sec. 5.B); any supported N (512 x 512:
 * a row and a column launch through the stream's scratch image, which steps rewrite anyway).
 * Synchronous: the value lands in *out.  Evaluation only, never part of a step. */
int ddh_strehl(ddh_state *s, const float *phi_true_dev, float *out);

/* Advance `count` states by one frame each: the states are grouped by grid size and path
 * (exec_path); each cluster-kernel group is one launch per 32 streams (plus one shared
 * post-step launch for its streams with the tile-phase prior or the sigma^2 M-step), each
 * staged group one launch sequence per chunk (ddh_set_staged_chunk); the groups run on
 * concurrent library-owned branches forked from and joined back into the stream of states[0],
 * which all states must share.  Each state appears at most once; frames as for ddh_step.  A
 * state's result does not depend on the other states in the batch (no arithmetic crosses
 * streams). */
int ddh_step_batch(ddh_state *const *states, const void *const *y_c64_dev, int count);

/* Batched step as a captured CUDA graph.  ddh_batch_create() records one step of every state
 * (any mix of N; all states on the stream and device of states[0], each at most once) into a
 * graph whose grid-size groups run on concurrent branches; the graph reads each stream's frame
 * through a device table of frame pointers owned by the batch.  ddh_batch_run() uploads the
 * table from `y_c64_dev` (count device pointers, 16-byte aligned, valid until the step has
 * run) on a library-owned copy stream, while the previous step may still run, and launches the
 * graph on that stream after the upload: one graph launch per time step.  Four instances of
 * the graph, each with its own table, take the steps in turn (a call waits on the host until
 * the step four calls earlier has finished).  The graph
 * holds each state's parameters as they were at creation: rebuild it after ddh_load.  The
 * batch does not own the states; free it before them. */
typedef struct ddh_batch ddh_batch;
int ddh_batch_create(ddh_batch **out, ddh_state *const *states, int count);
int ddh_batch_run(ddh_batch *b, const void *const *y_c64_dev);
int ddh_batch_free(ddh_batch *b);

/* ---- adjoint of one frame step (reverse mode through the EM iteration) -------------------
 * The paper defines no derivative; this is the chain rule through the step of ddh_step
 * (one EM iteration per frame, per-pixel phase, N <= 256: otherwise DDH_EINVAL).
 * Inputs (device, N*N float32 unless noted): the frame `y` (complex64, 16-byte aligned); the
 * state entering the frame (`r_prev`, `phi_prev`); the frame's ddh_step_trace output `trace`
 * recorded from that same state; the frame's output reflectance `r_new`; the gradients of a
 * scalar loss with respect to the outputs (`r_bar`, `phi_bar`).  Outputs: the gradients with
 * respect to the state entering the frame (`r_prev_bar`, `phi_prev_bar`, overwritten) and
 * `grads` (3 floats, ADDED to): dL/dprior_sigma, dL/dprior_p, dL/dnoise_var.  `workspace` is
 * caller-owned device memory of ddh_backward_workspace_bytes(N) bytes (16-byte aligned); the
 * call allocates nothing.  Enqueued on the state's stream; the state's own r, phi are untouched.
 * Non-differentiable points (floors, root-branch switches, zero surrogate differences) take
 * the one-sided or zero derivative. */
size_t ddh_backward_workspace_bytes(int n);
int ddh_step_backward(ddh_state *s, const void *y_c64_dev, const float *r_prev, const float *phi_prev,
                      const float *trace, const float *r_new, const float *r_bar, const float *phi_bar,
                      float *r_prev_bar, float *phi_prev_bar, float *grads, void *workspace,
                      size_t workspace_bytes);

/* K unrolled frame steps for reverse mode, looped inside the library (the per-frame calls of
 * ddh_step / ddh_step_trace / ddh_step_backward without a host round trip per frame).
 * ddh_unrolled_forward: from the state's current (r, phi), runs frames ys[0..K-1] (device,
 * complex64, 16-byte aligned) and stores the state entering each frame in r_ckpt[k],
 * phi_ckpt[k] (k = 0..K-1) and the final state in r_ckpt[K], phi_ckpt[K] (caller-owned device
 * images, N*N float32).  `traces` is NULL, or K caller-owned device buffers of
 * ddh_trace_floats(N) floats (8-byte aligned) that receive each frame's ddh_step_trace output.
 * The state ends in the final state.
 * ddh_unrolled_backward: given those checkpoints and the loss gradients with respect to the
 * final state (r_bar, phi_bar), writes the gradients with respect to the initial state
 * (r0_bar, phi0_bar) and ADDS the parameter gradients to grads[3] (as ddh_step_backward),
 * frame by frame in reverse.  With `traces` (the forward's) each frame's adjoint reads its
 * stored intermediates; with NULL each frame is first recomputed from its checkpoint into a
 * trace (less memory, one more step per frame); both give the same results bit for bit.
 * `workspace` is caller-owned device memory of ddh_unrolled_workspace_bytes(N) bytes (16-byte
 * aligned).  Both enqueue on the state's stream; the backward leaves the state at checkpoint
 * 0.  Requirements as ddh_step_backward (N <= 256, n_k = 1, per-pixel phase).  The paper has
 * no counterpart (training through the method is an extension). */
size_t ddh_unrolled_workspace_bytes(int n);
int ddh_unrolled_forward(ddh_state *s, int k_frames, const void *const *ys, float *const *r_ckpt,
                         float *const *phi_ckpt, float *const *traces);
int ddh_unrolled_backward(ddh_state *s, int k_frames, const void *const *ys, const float *const *r_ckpt,
                          const float *const *phi_ckpt, const float *const *traces, const float *r_bar,
                          const float *phi_bar, float *r0_bar, float *phi0_bar, float *grads, void *workspace,
                          size_t workspace_bytes);

/* Allocation-free variant of ddh_step_backward (the paper has no counterpart; this is a
 * library service).  Same arguments and results without the workspace: the scratch is a
 * static device array inside the library, 1796 KiB, present on every device that loads the
 * library until the process exits, sized for grids up to 128 x 128 (larger grids return
 * DDH_EINVAL with a message in ddh_last_cuda_error).  It is meant for callers that must not
 * allocate device memory while they run, such as a real-time control loop where cudaMalloc's
 * unbounded latency and possible device-wide synchronisation would break the frame deadline,
 * or a host whose device memory is fully budgeted up front.  The call itself never calls
 * cudaMalloc or cudaFree.  The first call on a device looks up the array's device address
 * (with that device current) and caches it per device and CUDA context (a call after a device
 * reset, in the new context, looks it up again); make that first call before any stream
 * capture.  Every call shares the one array, and each call initialises what it reads; calls
 * whose work overlaps on the GPU (other streams, other threads) race on it, so serialise them.
 * Argument checks are those of ddh_step_backward; each DDH_EINVAL sets a message. */
int ddh_step_backward_noalloc(ddh_state *s, const void *y_c64_dev, const float *r_prev, const float *phi_prev,
                              const float *trace, const float *r_new, const float *r_bar, const float *phi_bar,
                              float *r_prev_bar, float *phi_prev_bar, float *grads);

/* ---- streaming service: native continuous-batching scheduler -------------------------------
 * Sensors are admitted against a device-memory budget and keep their state resident; frames
 * are queued per sensor; a scheduler (a library thread after ddh_service_start, or each
 * ddh_service_poll call otherwise) resolves finished batches and launches the next queued
 * frame of every sensor that has one, as one ddh_step_batch, without waiting for batches still
 * running (at most `max_in_flight`; when a batch starts is decided by ddh_sched_pick
 * below).  A batch holds at most one frame per sensor; a sensor's
 * next frame may go into a later batch while its previous one still runs, since batches
 * execute in order on the service's stream.  A sensor's results do not depend on which
 * other sensors share its launches.  The paper has a frame loop per sensor
 * (Fig. 1); the multi-sensor service around it is this library's. */
#define DDH_SERVICE_PER_FRAME_LAUNCH 1u /* comparison mode: one ddh_step launch per frame */
typedef struct ddh_service ddh_service;
typedef struct ddh_completion {
  uint64_t tag;         /* the caller's tag from ddh_service_submit */
  int sensor;           /* sensor id */
  int64_t frame_index;  /* frames completed by this sensor, this one included */
  double arrival_s;     /* arrival time (ddh_service_now() clock) */
  double done_s;        /* time the scheduler saw the frame's batch complete */
} ddh_completion;
/* Create a service on `cuda_stream` (a non-default cudaStream_t; every admitted state is bound
 * to it).  mem_budget_bytes 0 = free device memory at creation minus 1 GiB. */
int ddh_service_create(ddh_service **out, void *cuda_stream, size_t mem_budget_bytes, int max_in_flight,
                       unsigned flags);
/* Device bytes one admitted state of grid n holds (r, phi, staging, status); 0 if n invalid. */
size_t ddh_state_bytes(int n);
/* Admit sensor `sensor_id` (unique) with parameters `p`: DDH_EBUDGET if its state would
 * exceed the budget.  Release frees the state once its queued and running frames are done. */
int ddh_service_admit(ddh_service *s, int sensor_id, const ddh_params *p);
int ddh_service_release(ddh_service *s, int sensor_id);
/* The sensor's state (for ddh_phase / ddh_reflectance between frames); NULL if unknown. */
ddh_state *ddh_service_state(ddh_service *s, int sensor_id);
/* Queue one frame (device pointer, caller-owned, valid until its completion is returned).
 * arrival_s < 0 stamps the current time. */
int ddh_service_submit(ddh_service *s, int sensor_id, const void *y_c64_dev, double arrival_s, uint64_t tag);
/* Return up to max_out completions in the order of their batches; drives one scheduler
 * iteration first when no library thread runs.  Returns a latched scheduler error if any. */
int ddh_service_poll(ddh_service *s, ddh_completion *out, int max_out, int *n_out);
int64_t ddh_service_pending(ddh_service *s); /* queued + running + unreturned frames */
int ddh_service_stats(ddh_service *s, int64_t *batches, int64_t *frames, size_t *used_bytes);
double ddh_service_now(void);                /* monotonic clock in seconds */
int ddh_service_start(ddh_service *s);      /* run the scheduler on a library thread */
int ddh_service_stop(ddh_service *s);
int ddh_service_free(ddh_service *s);        /* stops, waits for the stream, frees the states */

/* The service's batch-formation policy as a pure host function (no CUDA; the scheduler calls it
 * every iteration, and it can be exercised on its own, e.g. in a simulation).  Input: per
 * admitted sensor the number of queued frames and the arrival time (ddh_service_now clock) of
 * the oldest one; the number of the service's batches on the device and its limit.  Output:
 * pick[i] = 1 for the sensors whose next frame goes into a batch launched now; returns their
 * number (0: launch nothing now) or DDH_EINVAL.  Rule: nothing while `max_in_flight` batches
 * run; with no batch running, every sensor with a queued frame; behind a running batch only if
 * at least half of the sensors have a frame queued, or (flag DDH_SCHED_BACKLOG) some sensor has
 * two or more queued (its frames arrive faster than batches complete, and it advances one
 * frame per batch), or (flag DDH_SCHED_AGE) some queued frame is at least `age_limit_s` old.
 * The paper has no counterpart (its loop serves one sensor). */
#define DDH_SCHED_BACKLOG 1u
#define DDH_SCHED_AGE 2u
typedef struct ddh_sched_sensor {
  int queued;              /* frames waiting in the sensor's queue */
  double oldest_arrival_s; /* arrival time of the oldest of them (unused when queued == 0) */
} ddh_sched_sensor;
int ddh_sched_pick(const ddh_sched_sensor *sensors, int count, int batches_in_flight, int max_in_flight,
                   double now_s, double age_limit_s, unsigned flags, unsigned char *pick);
/* Select the policy's optional rules (DDH_SCHED_* flags; default both, age limit 1 ms). */
int ddh_service_set_policy(ddh_service *s, unsigned flags, double age_limit_s);

/* FFT radix schedule used for grid size n on the current device (the autotuner's choice):
 * count of schedules, select one (affects later launches and later ddh_batch_create), query.
 * Schedules differ only in rounding. */
int ddh_fft_schedule_count(int n);
int ddh_set_fft_schedule(int n, int schedule);
int ddh_get_fft_schedule(int n);
/* Streams per launch chunk of the L2-staged kernels for grid size n (128, 256, 512) on the
 * current device, 1..64 (default 16): a batch's staged streams of one size run as consecutive
 * launch sequences of this many streams, so that one chunk's working images (about 2.6 MB per
 * 256^2 stream, 10 MB per 512^2 stream) stay in L2 between its stages.  Affects later launches
 * and later ddh_batch_create; results do not depend on it (every stream's arithmetic is its
 * own).  The autotuner's knob. */
int ddh_set_staged_chunk(int n, int chunk);
int ddh_get_staged_chunk(int n);
/* on = 1: on the current device, every later batched step (ddh_step_batch, ddh_batch_create)
 * runs all its L2-staged streams -- of every staged grid size -- as one persistent cooperative
 * launch per step (or a few, when more than 64 streams, differing n_k or, with a graph, streams
 * interleaved with cluster-kernel streams split it): the grid's blocks take the stages' work
 * items (stream, block) in turn, with a grid-wide barrier between stages.  Results are bit for
 * bit those of the chained launches (on = 0, the default; the autotuner picks).  A barrier wait
 * is bounded (200 ms of device time); if one expires, every stream of that launch reports
 * DDH_ETIMEOUT and its state is left part-way through the step (restore it from a checkpoint).
 * Single-stream steps always use the chained launches. */
int ddh_set_staged_persistent(int on);
int ddh_get_staged_persistent(void);

/* Unitary 2D DFT (Sec. 2, F) or its inverse (inverse != 0) of one N x N complex64 image,
 * device in/out (may alias), on `cuda_stream`.  N = 32 ... 256. */
int ddh_fft2(const void *in_c64_dev, void *out_c64_dev, int n, int inverse, void *cuda_stream);

/* Wait for the state's stream; return and clear any latched device error. */
int ddh_sync(ddh_state *s);
/* Diagnostic of the device-side failure path, with no fault: a kernel on the state's stream
 * waits on a device barrier that nothing completes, gives up after `limit_s` seconds of device
 * time (0 < limit_s <= 1) and latches the same timeout status the step kernel latches when its
 * frame copy does not arrive in time.  Synchronises; returns DDH_ETIMEOUT (the expected result,
 * status cleared) and leaves the state usable, or DDH_EINVAL / DDH_ECUDA. */
int ddh_selftest_wait(ddh_state *s, double limit_s);

/* Checkpoint: `buf` (host) receives ddh_checkpoint_bytes(N) bytes: params, frame index, r,
 * phi.  ddh_load restores a state with the same N. */
size_t ddh_checkpoint_bytes(int n);
int ddh_save(ddh_state *s, void *buf, size_t bytes);
int ddh_load(ddh_state *s, const void *buf, size_t bytes);

int ddh_free(ddh_state *s);
const char *ddh_strerror(int code);
const char *ddh_last_cuda_error(void);
int ddh_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DDH_H_ */
