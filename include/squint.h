/*
 * squint.h - C ABI of the Squint visual-SAC learner on one GB300 (sm_103a).
 *
 * The library runs the batched Soft Actor-Critic update of Squint
 * (Almuzairee & Christensen, "Squint: Fast Visual Reinforcement Learning for
 * Sim-to-Real Robotics", Algorithm 1) as hand-written CUDA kernels, k updates
 * per call captured in one CUDA graph, and batched actor inference for parallel
 * environments beside it.
 *
 * Conventions for every entry point:
 *   - Return value: SQUINT_OK (0) or a negative SQUINT_E* code; squint_strerror
 *     gives its text, squint_last_error a message for the calling thread.
 *     No C++ exception or abort crosses this boundary.
 *   - Pointers documented as "device" are CUDA global-memory addresses on the
 *     device that was current when the handle was created; "host" pointers are
 *     ordinary CPU memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - Ownership: caller-owned buffers stay caller-owned and must stay valid
 *     until the work that reads them has completed on the given stream.
 *     Everything the library allocates is released by squint_destroy.
 *   - A CUDA failure inside a call returns SQUINT_ECUDA and marks the handle
 *     failed (sticky): later calls on it return SQUINT_ESTATE.
 */
#ifndef SQUINT_H
#define SQUINT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SQUINT_OK 0
#define SQUINT_EINVAL (-1)   /* bad argument or configuration */
#define SQUINT_ENOMEM (-2)   /* device allocation failed or memory budget exceeded */
#define SQUINT_ECUDA (-3)    /* a CUDA call failed (handle becomes failed) */
#define SQUINT_ETIMEOUT (-4) /* a bounded wait ran out */
#define SQUINT_EAGAIN (-5)   /* not ready yet / no capacity right now */
#define SQUINT_ESTATE (-6)   /* call not valid in the handle's current state */

#define SQUINT_MAX_CONV 8
#define SQUINT_MAX_HIDDEN 4

/* Arithmetic of the update's contractions (convs and linear layers).
 * Softmax, the atom projection, LayerNorm statistics, Adam and polyak are FP32
 * in every mode. */
#define SQUINT_PREC_FP32 0   /* plain FP32 CUDA-core kernels */
#define SQUINT_PREC_BF16 1   /* BF16 operands, FP32 accumulation (tensor cores) */
#define SQUINT_PREC_FP8 2    /* as BF16, with the forward linear layers in e4m3 (per-tensor
                                scales, FP32 accumulation); backward and convs stay BF16 */
#define SQUINT_PREC_MXFP8 3  /* as FP8, with MX block scales (one power of two per 32
                                elements of K of each row of both operands, see
                                squint_op_quantize_mxfp8) instead of per-tensor scales */

/*
 * Learner configuration (plain data, copied at creation).
 * Sizes follow the paper: squint = area downsampling of the rendered frame by
 * an integer factor (Sec. IV "Resolution Squinting"); a conv encoder shared by
 * actor and critic with per-head one-layer projections (Sec. IV "Encoder Design
 * Choices"); LayerNorm after every hidden linear layer (Sec. IV "Normalization");
 * a C51 critic on `atoms` atoms in [v_min, v_max] (Sec. IV "Critic Design
 * Choices"); two critics averaged in the target (Alg. 1); UTD updates per call.
 */
typedef struct {
    int32_t obs_c, obs_h, obs_w;     /* rendered frame, uint8 NCHW in the ring */
    int32_t squint_f;                /* area-downsampling factor (obs_h % squint_f == 0) */
    int32_t shift_pad;               /* random-shift pad p: crops at offsets in [0, 2p] */
    int32_t proprio_dim, action_dim;
    int32_t conv_layers, conv_ch;    /* valid 3x3 convs, ReLU after each.  conv_layers = 0:
                                        state-based SAC (Sec. VII, Fig. 6 left): no image and
                                        no encoder, the heads read the proprio_dim-wide state
                                        (>= 1); needs proj_dim = 0; obs_c, obs_h, obs_w,
                                        squint_f, shift_pad and conv_ch are then ignored */
    int32_t conv_stride[SQUINT_MAX_CONV];
    int32_t proj_dim;                /* 0: flatten straight into the heads */
    int32_t n_hidden;                /* hidden layers per MLP */
    int32_t hidden[SQUINT_MAX_HIDDEN];
    int32_t n_critics;               /* must be 2 */
    int32_t atoms;
    int32_t batch;
    int32_t policy_freq;             /* actor step when (update_idx + 1) % policy_freq == 0 */
    int32_t precision;               /* SQUINT_PREC_* */
    int32_t max_k;                   /* largest k accepted by squint_update */
    int32_t critic_kind;             /* 0: categorical C51 critic (Squint); 1: MSE critic with
                                        a scalar output (Eq. 2) */
    int32_t cdq;                     /* 0: average of the two critics (Squint); 1: clipped double
                                        Q, the smaller per sample, in the target and the actor */
    int32_t recompute_chunk;         /* 0: keep encoder activations; n > 0: BF16 tensor-core
                                        encoder only: run it in chunks of n images (rounded up
                                        to the weight gradient's images per CTA), keep only the
                                        features, recompute activations in the backward;
                                        results are bit-identical to n = 0 */
    double v_min, v_max, gamma, lr, tau, init_alpha;
    double target_entropy;           /* NaN: -action_dim */
    double ln_eps, log_std_min, log_std_max, adam_b1, adam_b2, adam_eps;
    uint64_t seed;                   /* Philox4x32-10 key for init and every draw */
} squint_config;

/* Replay ring (caller-owned device memory; the library only reads it).
 * Slot i holds the transition (o_i, s_i, a_i, r_i, d_i); its next observation is
 * slot (i + 1) mod n (Alg. 1 stores (o_t, s_t, a_t, r_t, o_{t+1}, s_{t+1})). */
typedef struct {
    const uint8_t* obs;      /* device [n, obs_c, obs_h, obs_w] uint8 (NULL if conv_layers = 0) */
    const float* proprio;    /* device [n, proprio_dim] */
    const float* action;     /* device [n, action_dim] in [-1, 1] */
    const float* reward;     /* device [n] */
    const uint8_t* done;     /* device [n], 0 or 1 */
    int64_t n;               /* slots, >= 2 */
} squint_replay;

/* Per-update diagnostics (one entry per update of a call). */
typedef struct {
    float critic_loss;   /* sum over critics of the batch-mean cross entropy */
    float actor_loss;    /* mean(alpha log pi - mean_i Q_i) (min_i with cdq); NaN when the actor did not step */
    float alpha_loss;    /* -alpha * mean(log pi + target_entropy) */
    float alpha;         /* temperature after the step */
    float q_mean;        /* mean over critics and batch of the online Q(s_t, a_t) */
    float entropy;       /* -mean log pi at s_t */
    int64_t update_idx;  /* index of this update (0-based, since creation) */
} squint_update_stats;

typedef struct squint_handle squint_handle;

/* ------------------------------------------------------------------ lifecycle */

/* Fill `cfg` with a named preset: "small_b32", "train_b512", "tiny_b8". */
int squint_config_preset(const char* name, squint_config* cfg);

/* Number of FP32 values in the canonical flat parameter layout of `cfg`:
 * encoder convs (w [co,ci,3,3], b), critic projection (w [d,f], b, ln g, ln b),
 * each critic's MLP (fc w [out,in], b, ln g, ln b per hidden layer; output fc),
 * actor projection, actor MLP (output 2*action_dim: mean, raw log-std), log_alpha.
 * Returns -1 for an invalid configuration. */
int64_t squint_param_count(const squint_config* cfg);

/* Create a learner on the current CUDA device.  Parameters are initialised from
 * cfg->seed (uniform +-1/sqrt(fan_in), LayerNorm 1/0, log alpha0), targets copy
 * the critics, Adam moments are zero.  `ring` may be NULL (inference only). */
int squint_create(const squint_config* cfg, const squint_replay* ring, squint_handle** out);

/* Replace the replay ring (pointers only; contents are read at update time).  A ring
 * with other pointers or another size drops the captured update graphs (after waiting
 * for the device): the next squint_update of each k captures again. */
int squint_set_replay(squint_handle* h, const squint_replay* ring);

/* Release everything the handle owns; waits for its own streams.  NULL is a no-op. */
int squint_destroy(squint_handle* h);

/* ------------------------------------------------------------------ hot path */

/*
 * Run k consecutive SAC updates (Alg. 1, inner loop; UTD k) on `stream`.
 * Each update: draw a minibatch of `batch` slots, random-shift and squint o_t and
 * o_{t+1}, encode both, build the C51 target from the averaged target critics,
 * step critics + encoder (Adam), step log alpha, step the actor on stop-gradient
 * features (every policy_freq updates), polyak-average the target critics.
 * The first call with a given k captures the k updates as one CUDA graph; later
 * calls replay it.  1 <= k <= cfg.max_k.
 * stats: NULL, or host array of k entries; when given the call waits for the
 * stream and fills it.  Returns SQUINT_ESTATE if no replay ring is set.
 */
int squint_update(squint_handle* h, int k, squint_update_stats* stats, void* stream);

/*
 * Same k updates issued as individual kernel launches (no graph).  Produces the
 * same result bit for bit; used to check the graph and for profiling.
 */
int squint_update_eager(squint_handle* h, int k, squint_update_stats* stats, void* stream);

/*
 * squint_update (the same k updates, Alg. 1 inner loop, as one graph) without waiting:
 * when stats is given, the stream itself copies the k entries there after the updates,
 * so the call returns at once and a training loop can issue the next call (and the
 * copies of new transitions) before it reads these statistics.  stats: NULL, or host
 * memory for k entries that the caller has page-locked (cudaMallocHost or
 * cudaHostRegister; pageable memory is rejected with SQUINT_EINVAL); its contents are
 * valid once the stream has passed this call (cudaStreamSynchronize, or an event the
 * caller records after it), and the caller must not reuse the buffer before then.
 * A bounded device wait that ran out is reported by the next call that waits
 * (squint_update with stats, squint_update_check).  Returns as squint_update otherwise.
 */
int squint_update_async(squint_handle* h, int k, squint_update_stats* stats, void* stream);

/*
 * Waits for `stream` and reports whether a bounded device wait of the updates issued
 * so far ran out (SQUINT_ETIMEOUT, and the handle is marked failed) or not (0).
 */
int squint_update_check(squint_handle* h, void* stream);

/* ------------------------------------------------------------------ measurement */

/* Kernel nodes in the graph captured for k updates (0 if none captured yet). */
int64_t squint_graph_kernel_count(squint_handle* h, int k);

/* Device bytes the learner allocated at creation (parameters, optimiser state,
 * activations, workspaces; not the caller's ring, not inference buffers).  0 for NULL. */
int64_t squint_device_bytes(squint_handle* h);

/*
 * One update issued eagerly on `stream` with a CUDA event at every phase
 * boundary; ms[i] receives the device time of phase i (see squint_phase_name)
 * and *n_phases their number (at most cap are written).  Waits for the stream.
 */
int squint_profile_update(squint_handle* h, float* ms, int cap, int* n_phases, void* stream);
/* Name of phase i of squint_profile_update, or NULL. */
const char* squint_phase_name(int i);

/*
 * One update issued eagerly on `stream` with every kernel launched in order (no
 * concurrent branches) and timed by its own CUDA events; launches are grouped by
 * kernel class.  For class i < *n (at most cap written): names + 32 i receives its
 * NUL-terminated name, launches[i] its launch count, ms[i] its total device time,
 * work[i] the algorithmic work of those launches and unit[i] its unit (0: FLOP,
 * 1: bytes of DRAM-level traffic the class needs at minimum).  Waits for the stream.
 */
int squint_profile_kernels(squint_handle* h, int cap, char* names, int* launches, float* ms, double* work, int* unit,
                           int* n, void* stream);

/*
 * A timeline of one update as the timed graph runs it (its concurrent branches kept):
 * every launch bracketed by CUDA events.  For launch i < *n (at most cap written, in
 * issue order): names + 32 i its kernel class (NUL-terminated), lanes[i] the branch it
 * ran on (0: the main stream; 1 ..: the learner's side streams), t0[i] and t1[i] its
 * start and end in ms after the update's start.  The event pairs themselves add a
 * little time per launch.  Waits for the stream.
 */
int squint_trace_update(squint_handle* h, int cap, char* names, int* lanes, float* t0, float* t1, int* n,
                        void* stream);

/* ------------------------------------------------------------------ inference */

/* One actor query: n environments of one group (Alg. 1, "Sample a_t ~ pi"). */
typedef struct {
    uint64_t group_id;       /* caller's tag */
    int32_t n;               /* environments (rows), >= 1 */
    int32_t mode;            /* 0: sample a = tanh(mu + sigma eps); 1: mean tanh(mu) */
    uint64_t rng_key;        /* noise of row r = Philox block (r, act stream, rng_key) */
    const uint8_t* obs;      /* device [n, obs_c, obs_h, obs_w] uint8 render-resolution frames
                                (NULL if conv_layers = 0) */
    const float* proprio;    /* device [n, proprio_dim] */
    float* actions;          /* device [n, action_dim] output in (-1, 1) */
} squint_act_request;

/*
 * Actions for n_reqs requests as one ragged batch on `stream` (squint without
 * shift, encoder, actor projection, actor MLP, tanh-Gaussian head).  Uses the
 * inference snapshot of the actor (see squint_refresh_policy); a row's result
 * does not depend on the other rows of the batch.
 */
int squint_act(squint_handle* h, const squint_act_request* reqs, int n_reqs, void* stream);

/*
 * Copy the current encoder + actor weights into the inference snapshot, ordered
 * after the work already queued on `stream` (typically the update stream).
 * Inference launched afterwards sees a consistent snapshot; the snapshot version
 * increments by one per refresh.
 */
int squint_refresh_policy(squint_handle* h, void* stream);

/* ------------------------------------------------------------------ serving loop */

/*
 * Continuous-batching server for actor queries (Alg. 1, "Sample a_t ~ pi": batched
 * inference for the parallel environments).  A host scheduler thread keeps up to
 * `slots` batches in flight (3 by default; SQUINT_SERVE_SLOTS=1..4 in the environment
 * at start), each slot with its own activation arena and its own stream at the
 * device's highest priority.  Whenever a slot is free it admits queued requests in
 * arrival order up to the slot's rows and launches them as one ragged batch, so
 * requests that arrive while others run are admitted as slots free up and their work
 * overlaps the batches still on the GPU.  Admission by memory: the arenas are
 * allocated at start and hold at most mem_budget_bytes (and at most 90% of the
 * device's free memory); max_rows bounds a batch (fewer rows per slot, or fewer
 * slots, when the budget asks for it).  A row's result does not depend on the other
 * requests of its batch.
 */
int squint_serve_start(squint_handle* h, int max_rows, size_t mem_budget_bytes);
/* Queue a request (buffers must stay valid until it completes); *ticket receives its id.
 * SQUINT_EAGAIN if the queue is full, SQUINT_EINVAL if it can never be admitted (more
 * rows than a slot holds), SQUINT_ESTATE if the server is not running. */
int squint_serve_submit(squint_handle* h, const squint_act_request* req, uint64_t* ticket);
/* What a completed request reports. */
typedef struct {
    double latency_us;        /* submit to completion: queueing on the host until its batch was
                                 launched, plus the batch's device time from its launch marker
                                 to its completion event */
    int64_t policy_version;   /* policy snapshot the batch read */
    double device_begin_us;   /* the batch's launch marker and completion on the device, in */
    double device_end_us;     /* microseconds from the server's start */
    int32_t slot;             /* the slot (arena and stream) that ran it */
    int32_t batch_rows;       /* rows of its batch */
} squint_serve_result;
/* Wait up to timeout_us (0 = poll) for a ticket.  SQUINT_OK when done (*out filled if not
 * NULL); SQUINT_EAGAIN if not yet; SQUINT_ESTATE if the server stopped without it. */
int squint_serve_poll_ex(squint_handle* h, uint64_t ticket, int64_t timeout_us, squint_serve_result* out);
/* The same, reporting only the latency and the policy version (either may be NULL). */
int squint_serve_poll(squint_handle* h, uint64_t ticket, int64_t timeout_us, double* latency_us,
                      int64_t* policy_version);
/* Slots, rows per slot and the device bytes the slots' arenas hold. */
int squint_serve_info(squint_handle* h, int* slots, int* slot_rows, int64_t* arena_bytes);
/* Stop the scheduler after the queued and in-flight work completes; waiting pollers
 * of tickets it never completes return SQUINT_ESTATE.  Safe while other threads submit
 * or poll. */
int squint_serve_stop(squint_handle* h);

/* ------------------------------------------------------------------ state */

/* Parameters in the canonical flat FP32 layout (host buffers of squint_param_count values). */
int squint_get_params(squint_handle* h, float* host, int64_t n);
int squint_set_params(squint_handle* h, const float* host, int64_t n);

/* Full learner state: params, Adam m and v, target critics, step counters,
 * update index.  Call with host == NULL to query *bytes. */
int squint_get_state(squint_handle* h, void* host, size_t* bytes);
int squint_set_state(squint_handle* h, const void* host, size_t bytes);

/* Copy a named internal buffer of the last update to host (tests, debugging):
 * "idx" int32[B], "nxt" int32[B], "shift_t"/"shift_t1" int32[B,2] (dx, dy),
 * "sums_t"/"sums_t1" uint16[B,C,Hs,Ws] box sums, "x_t"/"x_t1" f32[B,C,Hs,Ws],
 * "m" f32[B,K] projected target, "logits" f32[E,B,K], "logits_target" f32[E,B,K],
 * "logp_next" f32[B], "logp_t" f32[B], "a_next" f32[B,A], "a_pi" f32[B,A],
 * "grads" f32[param_count] (critic group from the critic step, actor group from
 * the actor step), "z_t" f32[B,F], "conv0".."conv7" f32[B,ch,oh,ow] (conv layer l's
 * output after its ReLU, o_t images; learners that keep FP32 conv planes), "dconv0"
 * f32[B,ch,oh,ow] (gradient at the first conv's pre-activation, after the ReLU mask;
 * FP32 planes) or "dconv0_phwc" bf16 (the same in padded HWC: per image (oh+4)(ow+4)
 * pixels of 32 channels, pixel (y,x) at (y+2)(ow+4)+x+2; tensor-core encoder without
 * recompute).  *bytes in: capacity, out: size; SQUINT_EINVAL for a name this learner
 * does not keep. */
int squint_debug_tensor(squint_handle* h, const char* name, void* host, size_t* bytes);

/* Failure-detection settings (tests).  Every wait of the tensor-core kernels on an
 * mbarrier is bounded: past its limit the waiting thread records a code in the
 * handle's device error word and gives up, the CTA waits (bounded) for the copies it
 * still has in flight, frees its tensor memory and returns; squint_update with
 * statistics then reports SQUINT_ETIMEOUT and the handle is failed.  Settings:
 * "wait_cycles" = clock cycles a wait of the update's tensor-core GEMMs may take
 * (0: the default, about 2 s); "stall_gemm_loads" = 1 makes those GEMMs issue no
 * operand loads, so their first operand wait runs out with nothing in flight (the
 * way a test makes a wait run out without faulting anything).  Captured update
 * graphs are dropped when a setting changes.  SQUINT_EINVAL for an unknown name or
 * value. */
int squint_set_debug(squint_handle* h, const char* name, int64_t value);

/* ------------------------------------------------------------------ errors */

/* sizeof of an ABI struct by name ("squint_config", "squint_replay",
 * "squint_update_stats", "squint_act_request"); 0 for an unknown name.
 * Lets a binding check its struct layouts against the compiled library. */
size_t squint_struct_size(const char* name);

const char* squint_strerror(int code);
/* Message of the last failure on the calling thread ("" if none). */
const char* squint_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SQUINT_H */
