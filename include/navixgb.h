/*
 * navixgb.h -- C ABI of the GB300-native batched MiniGrid environment step
 * (NAVIX, arXiv 2407.19396).
 *
 * The environment is the paper's tuple M = (h, w, T, O, A, R, d, O, R, gamma,
 * P) (Section 3.2.1): grid height/width, a timeout T (max_steps), the
 * symbolic_first_person / rgb_first_person observation functions (Table 4),
 * the Markovian rewards R1-R3 (Table 8, Table 5), the terminations of
 * Table 6, the intervention and transition systems (Table 3, Appendix A) and
 * the timestep/autoreset protocol (Section 3.2.2, Code 1).  The batching over
 * environments is the paper's vmap (Code 3); nx_rollout is the jitted scan of
 * Code 2 as persistent, graph-captured chunks.
 *
 * Conventions shared by every call:
 *   - All functions return nx_status (0 = NX_OK, < 0 = error).  Nothing in
 *     the library aborts, exits or traps; argument errors are reported
 *     synchronously, device-side problems through nx_sync().
 *   - A context is bound to one CUDA stream (the one given at creation); all
 *     work is enqueued on it and is asynchronous to the host unless the call
 *     says otherwise.  Calls on one context must not run concurrently from
 *     several host threads.
 *   - Device pointers passed in are owned by the caller and must stay valid
 *     until the enqueued work has finished.  Memory the library allocates is
 *     owned by the context and released by nx_destroy().
 *   - Cell codes: entity 0 unseen, 1 empty, 2 wall, 3 floor, 4 door, 5 key,
 *     6 ball, 7 box, 8 goal, 9 lava, 10 agent; colour 0 red, 1 green, 2 blue,
 *     3 purple, 4 yellow, 5 grey; door state 0 open, 1 closed, 2 locked.
 *     Directions 0 east (+x), 1 south (+y), 2 west, 3 north.  Actions 0 left,
 *     1 right, 2 forward, 3 pickup, 4 drop, 5 toggle, 6 done.
 *   - Randomness: every draw is word 0 of Philox4x32-10 (Salmon et al.,
 *     SC'11) with key (seed lo, seed hi) and counter (env index, episode,
 *     step, purpose << 24 | draw); a bounded draw in [0, n) is
 *     (x * n) >> 32.  Purposes: 1 layout, 2 ball move, 3 random action (the
 *     episode word is then 0xFFFFFFFF and the step word is the number of
 *     step calls since nx_reset).  Results therefore do not depend on the
 *     launch configuration, on the GPU count or on the other envs in a batch.
 */
#ifndef NAVIXGB_H
#define NAVIXGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t nx_status;
enum {
    NX_OK = 0,
    NX_PENDING = 1,          /* nx_poll: the request has not finished */
    NX_E_INVAL = -1,         /* invalid argument */
    NX_E_NOMEM = -2,         /* an allocation failed */
    NX_E_CUDA = -3,          /* a CUDA runtime call failed (see nx_last_error) */
    NX_E_TIMEOUT = -4,       /* a bounded host wait expired */
    NX_E_DEVICE_CHECK = -5,  /* a device-side consistency check fired */
    NX_E_BUDGET = -6,        /* a serving request can never fit the HBM budget */
    NX_E_STATE = -7,         /* call out of order (e.g. step before reset) */
    NX_E_CANCELED = -8       /* a serving request withdrawn by nx_cancel */
};

/* environment families of Table 8; the crossings take their number of
 * rivers as the descriptor's variant (0..nx_max_variant), DistShift its
 * layout (variant 0: DistShift1, 1: DistShift2).  KeyCorridor S{s}R{R} has
 * size 3(s-1)+1 (7, 10, 13, 16, 19 for s = 3..7) and variant R - 1 (0..2);
 * its grid of (s-1)R+1 rows is held in the square with wall rows below,
 * which leaves the first-person views and the rules those of the smaller
 * grid (the fully observable views show the wall rows).  GoToDoor has a
 * mission (the colour of one of its four doors, nx_out.mission) and ends
 * with reward 1 when the done action is taken facing that door
 * (on_door_done, Tables 5 and 6). */
enum {
    NX_EMPTY = 0, NX_DOORKEY = 1, NX_FOURROOMS = 2, NX_LAVAGAP = 3, NX_DYNOBS = 4, NX_EMPTY_RANDOM = 5,
    NX_LAVA_CROSSING = 6, NX_SIMPLE_CROSSING = 7, NX_GOTODOOR = 8, NX_DISTSHIFT = 9, NX_KEYCORRIDOR = 10
};
#define NX_N_FAMILIES 11
#define NX_NO_MISSION 255  /* the mission byte of a family without one */
/* observation bit flags (Table 4): RGB and RGB_FULL need the sprite atlas */
enum { NX_OBS_SYM = 1, NX_OBS_RGB = 2, NX_OBS_RGB_FULL = 4 };
/* action sources: a device buffer, the counter hash's uniform draw, or the
 * context's fused policy (nx_set_policy) */
enum { NX_ACT_BUFFER = 0, NX_ACT_RANDOM = 1, NX_ACT_POLICY = 2 };
/* reward functions: Markovian (Section 3.2.1, Table 5) or MiniGrid's Eq. 1 */
enum { NX_REWARD_MARKOV = 0, NX_REWARD_MINIGRID = 1 };
/* staging of the symbolic outputs in shared memory (tunable; never changes
 * results): the whole thread block's block of observations at once, or in
 * two halves (half the staging memory, so more envs stay resident) */
enum { NX_STAGE_AUTO = 0, NX_STAGE_FULL = 1, NX_STAGE_HALF = 2 };

#define NX_MIN_SIZE 5
#define NX_MAX_SIZE 19
#define NX_VIEW 7
#define NX_OBS_SYM_BYTES 147        /* 7 x 7 x 3 */
#define NX_OBS_RGB_BYTES 150528     /* 224 x 224 x 3 */
#define NX_ATLAS_TILES 401
#define NX_ATLAS_BYTES (401 * 3072) /* 401 tiles of 32 x 32 x 3 */
#define NX_AGENT_BYTES 32
#define NX_MAX_BALLS 4

typedef struct nx_env nx_env;
typedef struct nx_server nx_server;

/* One environment's shape: family, square grid side (height == width,
 * 5..19), timeout T (<= 0: the family default: DoorKey 10 S^2, FourRooms
 * 100, GoToDoor 5 S^2, KeyCorridor 30 s^2 for room side s, the others 4 S^2;
 * at most 65535), and the family's variant (the number
 * of rivers of a crossing family, 0 otherwise). */
typedef struct {
    int32_t family, height, width, max_steps, variant;
} nx_desc;

/* Creation options; nx_options_default() fills the defaults. */
typedef struct {
    uint32_t obs_flags;       /* NX_OBS_SYM | NX_OBS_RGB (default NX_OBS_SYM) */
    int32_t reward_mode;      /* NX_REWARD_MARKOV (default) or NX_REWARD_MINIGRID */
    float lava_reward;        /* reward on stepping into lava (default 0.0f; the paper's R2 uses -1) */
    int32_t n_balls;          /* Dynamic-Obstacles balls, 0..4 (default 4) */
    int32_t steps_per_launch; /* steps per persistent chunk in nx_rollout, 1..1024 (default 128) */
    int32_t autotune;         /* 1: time the launch shapes once and keep the fastest (default 1) */
    int32_t group_lanes;      /* lanes per env, 1/2/4/8/16/32; 0 = chosen by the library */
    int32_t envs_per_cta;     /* envs per thread block; 0 = chosen by the library */
    int32_t staging;          /* NX_STAGE_*; 0 = chosen by the library (used with group_lanes) */
    const uint8_t* atlas;     /* host sprite atlas, NX_ATLAS_BYTES (required with NX_OBS_RGB / _RGB_FULL) */
    /* optional device allocator (e.g. a framework's caching allocator); NULL: cudaMallocAsync */
    void* (*alloc)(size_t bytes, void* user);
    void (*free)(void* ptr, void* user);
    void* alloc_user;
    /* global index of this context's env 0 in the draw counters (default 0):
     * contexts over disjoint index ranges reproduce one large batch exactly,
     * which is how a batch is split over GPUs */
    uint32_t env_index_base;
    int32_t variant;          /* nx_create only: the variant of every env (rivers of a crossing family) */
    /* Table 5's shaping terms, subtracted from every step's reward in this
     * order: action_cost for each action 0..5 (every action but done), then
     * time_cost (default 0 and 0; not applied to autoreset steps) */
    float action_cost;
    float time_cost;
    /* shared-memory slots of the step kernel sized for grids of this side
     * (0: chosen by the autotuner with the launch shape, else the largest
     * side of the batch); work items of larger grids then hold fewer envs.
     * Results never depend on it. */
    int32_t grid_side;
} nx_options;

/* Per-step outputs, device pointers owned by the caller; any may be NULL (not
 * written).  Shapes are [depth, n_envs, ...] row-major: obs_sym [.., 7, 7, 3]
 * uint8 laid out [view row vy][view column vx][entity, colour, state] with
 * the agent at (vx 3, vy 6) facing vy = 0 (symbolic_first_person, Table 4);
 * obs_rgb [.., 224, 224, 3] uint8 (rgb_first_person); reward [..] float32;
 * terminated / truncated [..] uint8 (0/1).  Step i of a call writes time
 * slot i % depth (depth <= 0 means 1).
 * The fully observable views of Table 4 (device rollouts only):
 * obs_full [.., full_side, full_side, 3] (symbolic: every cell's triple, row
 * y then column x, the agent's cell holding (10, 0, direction)), obs_cat
 * [.., full_side, full_side] (categorical: entity codes, the agent 10), both
 * zero beyond an env's grid; obs_cat_fp [.., 7, 7] (categorical_first_person:
 * the entity bytes of obs_sym).  full_side must be at least the largest grid
 * size (0: the largest grid size).  obs_rgb_full [.., 32 full_side,
 * 32 full_side, 3] (rgb: every cell's sprite, the agent drawn facing its
 * direction; needs NX_OBS_RGB_FULL at creation and full_side equal to the
 * largest grid size).
 * mission [..] uint8: the mission of the episode the slot's observation
 * belongs to (GoToDoor: the target door's colour index; NX_NO_MISSION for
 * the other families).  action [..] int8: the action of the step (drawn,
 * read from the buffer or chosen by the policy; an env that starts an
 * episode on that step ignores it). */
typedef struct {
    uint8_t* obs_sym;
    uint8_t* obs_rgb;
    float* reward;
    uint8_t* terminated;
    uint8_t* truncated;
    int32_t depth;
    int32_t full_side;
    uint8_t* obs_full;
    uint8_t* obs_cat;
    uint8_t* obs_cat_fp;
    uint8_t* obs_rgb_full;
    uint8_t* mission;
    int8_t* action;  /* [.., n] the action each step took (device rollouts only) */
} nx_out;

/* Launch shape in use (after autotuning); policy_* describe the fused-policy
 * launches (0 before nx_set_policy).  lean_family >= 0: rollouts of this
 * context with random actions, no action output and the Markov reward (and
 * no RGB or fully observable views) launch a step kernel compiled for such
 * calls -- for that one family, or for any family where it is
 * NX_N_FAMILIES -- on lean_grid_ctas CTAs; -1: every call runs the general
 * one. */
typedef struct {
    int32_t group_lanes, envs_per_cta, staging, n_items, grid_ctas, smem_bytes, steps_per_launch;
    int32_t n_envs, n_families;
    size_t state_bytes, device_bytes;
    int32_t policy_items, policy_ctas_per_sm, policy_grid_ctas, policy_smem_bytes;
    int32_t lean_family, lean_grid_ctas;
    int32_t grid_side;   /* the grid side the block's shared-memory slots are sized for */
} nx_info;

void nx_options_default(nx_options* opts);
/* Largest valid variant of a family at a size (the number of candidate
 * rivers of a crossing family: rows and columns 2, 4, .., size-3; 1 for
 * DistShift; 2 for KeyCorridor), 0 for the other families, -1 where the
 * family has no grid of that size (KeyCorridor off 7, 10, 13, 16, 19). */
int32_t nx_max_variant(int32_t family, int32_t size);

/* nx_create: one family and size for all n_envs environments (the paper's
 * make(id), Code 1, batched as in Code 3).  n_envs >= 1.  seed keys every
 * draw.  cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Allocates the device state (about 3 S^2 + 32 bytes per env) but does not
 * initialise it: call nx_reset before stepping.  NX_E_INVAL on bad
 * arguments, NX_E_NOMEM / NX_E_CUDA on allocation or device failures. */
nx_status nx_create(nx_env** env, int32_t family, int32_t size, int32_t n_envs, uint64_t seed,
                    const nx_options* opts, void* cuda_stream);

/* nx_create_mixed: one descriptor per environment (host array of n_envs).
 * Environments with equal descriptors should be contiguous: each maximal
 * run of equal descriptors is batched separately. */
nx_status nx_create_mixed(nx_env** env, const nx_desc* host_descs, int32_t n_envs, uint64_t seed,
                          const nx_options* opts, void* cuda_stream);

/* nx_reset: reset(key) of Section 3.2.2 for every env (episode 0), the step
 * counter of random actions restarts at 0.  Writes the initial observation
 * with reward 0 and both flags 0 (the paper's reward padding) into slot 0 of
 * out (out or any pointer in it may be NULL). */
nx_status nx_reset(nx_env* env, const nx_out* out);

/* nx_step: one step(timestep, action) of Code 1 for every env, with
 * autoreset: an env whose previous step terminated or truncated starts its
 * next episode instead (reward 0, flags 0, the action is ignored).
 * d_actions: device int8 [n_envs]; NULL draws uniform random actions (7, or
 * 3 in Dynamic-Obstacles).  Out-of-range actions are executed as no-ops and
 * set a sticky flag (nx_device_flags).  Step order inside one env: autoreset,
 * transition (Dynamic-Obstacles balls), intervention, reward/termination,
 * time/truncation, observation. */
nx_status nx_step(nx_env* env, const int8_t* d_actions, const nx_out* out);

/* nx_rollout: n_steps consecutive nx_step calls fused into persistent,
 * CUDA-graph-captured chunks of steps_per_launch steps (the jitted scan of
 * Code 2).  act_mode NX_ACT_RANDOM ignores d_actions_TN; NX_ACT_BUFFER reads
 * device int8 [n_steps, n_envs]; NX_ACT_POLICY chooses every action with the
 * context's policy from the env's current view (no RGB or fully observable
 * outputs then).  Step i writes slot i % traj->depth. */
nx_status nx_rollout(nx_env* env, int32_t n_steps, int32_t act_mode, const int8_t* d_actions_TN,
                     const nx_out* traj);

/* nx_rollout_per_family: the plain comparison form of nx_rollout -- the
 * same results, computed with one single-step launch per family per step
 * (state round-trips through HBM every step, no graph). */
nx_status nx_rollout_per_family(nx_env* env, int32_t n_steps, int32_t act_mode, const int8_t* d_actions_TN,
                                const nx_out* traj);

/* nx_rollout_host: nx_rollout with HOST buffers (pinned memory gives
 * overlap): actions are copied in and outputs copied back chunk by chunk on
 * the context stream; returns when the copies have finished.  host_actions_TN
 * is int8 [n_steps, n_envs] (ignored for NX_ACT_RANDOM); the host outputs are
 * [D, n_envs, ...] with D = host_traj->depth, step i written to host slot
 * i % D (depth <= 0, or >= n_steps: D = n_steps, one slot per step), so a
 * long rollout can stream through a bounded pinned ring; every slot ends
 * holding the last step written there, and nothing is written beyond the
 * D slots, whatever the chunk length (steps_per_launch).  Any output may be
 * NULL; the fully observable views and the action output are not available
 * here (NX_E_INVAL). */
nx_status nx_rollout_host(nx_env* env, int32_t n_steps, int32_t act_mode, const int8_t* host_actions_TN,
                          const nx_out* host_traj);

/* The fused policy + environment rollout (the PPO rollout pattern of
 * Section 4's batch-mode experiment, many agents each stepping its own
 * envs): an integer MLP evaluated on the tensor cores inside the step
 * kernel.  It maps each env's categorical first-person view x (49 entity
 * codes, Table 4) to one logit per action:
 *   h1[j] = clamp((sum_k w1[j][k] x[k] + b1[j]) >> shift1, 0, 255)
 *   h2[j] = clamp((sum_i w2[j][i] h1[i] + b2[j]) >> shift2, 0, 255)
 *   z[a]  = sum_i w3[a][i] h2[i] + b3[a]
 * (>> floors), takes the first largest z[a] over the family's actions, and
 * with an exploration draw below epsilon (of 2^32) the uniform random
 * action instead.  Env e (its global draw index) uses weight set
 * e / envs_per_agent.  Host arrays: w1 [n_agents][64][49], b1 [n_agents][64],
 * w2 [n_agents][64][64], b2 [n_agents][64], w3 [n_agents][7][64],
 * b3 [n_agents][7]; |bias| <= 2^22, shifts 0..24.  The policy runs 128 envs
 * per thread block: envs_per_agent is 16, 32 or 64 (each block then holds
 * 8, 4 or 2 weight sets, and every block of the context's work list must
 * start at a weight-set boundary) or at least 128 (a weight set must cover
 * whole blocks); NX_E_INVAL otherwise.  The weights are copied to the device
 * (the host arrays may be freed on return). */
typedef struct {
    int32_t n_agents, envs_per_agent;
    const int8_t* w1;
    const int32_t* b1;
    const int8_t* w2;
    const int32_t* b2;
    const int8_t* w3;
    const int32_t* b3;
    int32_t shift1, shift2;
    uint32_t epsilon;
} nx_policy;
nx_status nx_set_policy(nx_env* env, const nx_policy* policy);

/* State snapshot (checkpoint/resume).  Blocking.  Layout of the buffer:
 *   [0, 64)                header: "NXST", version 1, n_envs, gstep (u32 at 12),
 *                          grid pool bytes (u64 at 16), seed (u64 at 24)
 *   [64, 64 + 32 n)        per-env agent blocks, NX_AGENT_BYTES each:
 *       u8 x, y, dir, carry_ent, carry_col, done, invalid, n_balls;
 *       u16 t, max_steps; u32 episode; u8 ball_x[4], ball_y[4];
 *       u8 family, size, mission (NX_NO_MISSION without one), reserved;
 *       u32 grid_offset: the low 32 bits of the env's byte offset in the pool
 *   [64 + 32 n, end)       grid pool: the envs in order, each one's three
 *                          planes of size*size bytes (entity, colour, state,
 *                          row-major y * size + x) right after the previous
 *                          env's, so env i starts at the sum of 3 size^2 over
 *                          the envs before it (pools may exceed 4 GiB).
 * nx_set_state accepts only a snapshot of a context with the same
 * descriptors, and only states the steps can reach: every index inside
 * its env's grid, cell and carried codes in range, and each
 * Dynamic-Obstacles ball in the grid's interior (1..size-2: balls are
 * placed there and only move to empty cells); anything else is NX_E_INVAL
 * and nothing is applied. */
size_t nx_state_bytes(const nx_env* env);
nx_status nx_get_state(nx_env* env, void* host_buf, size_t bytes);
nx_status nx_set_state(nx_env* env, const void* host_buf, size_t bytes);

/* Waits (bounded by timeout_s, <= 0: no bound) for the context's stream and
 * surfaces deferred device errors: NX_E_TIMEOUT, NX_E_CUDA or
 * NX_E_DEVICE_CHECK. */
nx_status nx_sync(nx_env* env, double timeout_s);
/* Sticky device flags (bit 0: an out-of-range action was seen; bit 1: an
 * internal bounds check fired).  Blocking. */
nx_status nx_device_flags(nx_env* env, uint32_t* flags);
nx_status nx_get_info(const nx_env* env, nx_info* info);

/* Kernel instrumentation.  nx_profile_begin starts recording a CUDA event
 * pair on the context stream around every step-kernel launch (a captured
 * chunk counts as one launch: its step kernel plus the two-word counter
 * update).  nx_profile_end waits for the stream and returns the summed
 * device time of those launches in milliseconds and their count.
 * nx_launch_counts returns the cumulative number of step-kernel launches and
 * of all kernels this context has enqueued (graph replays count their
 * nodes); it never blocks. */
/* ------------------------------------------------------------------------
 * Serving: continuous batching of rollout requests (the paper's batch mode,
 * Section 4.2 and Appendix B, as a request loop).  A request is a fresh batch
 * of n_envs envs of one family and size, reset to episode 0 and stepped
 * `horizon` times with uniform random actions keyed by (request seed,
 * request-local env index, request-local step), exactly as nx_create +
 * nx_reset + nx_rollout(horizon, NX_ACT_RANDOM) would.  Requests that arrive
 * while others run are admitted (strictly first come, first served) as soon
 * as their device memory fits in the server's fixed HBM budget; all admitted
 * requests advance together in each chunk (one persistent launch per launch
 * shape), so results do not depend on what else is in flight.
 */
#define NX_REQ_DIGEST 1u  /* nx_request.flags: compute nx_result.digest (else it is 0) */

typedef struct {
    int32_t family, size, n_envs, horizon;  /* size 5..19, n_envs >= 1, horizon >= 1 */
    int32_t variant;                        /* the family's variant (rivers of a crossing family) */
    uint32_t flags;                         /* NX_REQ_DIGEST or 0; other bits: NX_E_INVAL */
    uint64_t seed;
    /* optional host outputs, written when the request finishes:
     * returns [n_envs] float32 (sum of rewards over the horizon, in step
     * order) and final_obs [n_envs, 7, 7, 3] uint8 (the last step's view) */
    float* returns;
    uint8_t* final_obs;
} nx_request;

typedef struct {
    nx_status status;          /* NX_OK when finished */
    double t_submit, t_start, t_done;  /* seconds on the server's steady clock */
    uint64_t digest;           /* 64-bit digest of every per-step output (see below), 0 without NX_REQ_DIGEST */
    uint64_t env_steps;        /* n_envs x horizon */
    uint32_t episodes;         /* episodes that ended (terminated or truncated) */
} nx_result;
/* Digest (requests with NX_REQ_DIGEST; the folds cost the kernel more than
 * the step itself): per env, h = 0; for the reset record and then every step record
 * fold the 49 view cells as words (ent | col << 8 | st << 16), the reward's
 * float32 bits and (terminated | truncated << 8), each by
 * h = (h ^ w) * 0x100000001B3 (mod 2^64); the request digest folds the
 * per-env values (low word, then high word, env by env) the same way. */

typedef struct {
    uint64_t submitted, finished, rejected, env_steps, chunks;
    double busy_s;             /* time with at least one request on the GPU */
    size_t budget_bytes, in_use_bytes, peak_bytes;
    uint64_t canceled;         /* requests withdrawn by nx_cancel */
} nx_server_stats;

/* nx_server_create: hbm_budget_bytes (1 MiB .. 1 TiB) is allocated once, up
 * front, and every admitted request's state and outputs are carved from it.
 * opts: steps_per_launch is the chunk length (latency vs launch overhead),
 * group_lanes / envs_per_cta / staging fix one launch shape for every
 * request (0: 1 lane per env, 128 envs per block, half staging, with
 * requests of at most 64 envs run at 16 lanes per env on a second stream
 * beside them), reward options apply to every request; obs_flags must be
 * NX_OBS_SYM. */
nx_status nx_server_create(nx_server** server, size_t hbm_budget_bytes, const nx_options* opts, void* cuda_stream);
/* nx_submit: queue a request; NX_E_BUDGET if it can never fit the budget,
 * NX_E_INVAL on bad arguments.  The host output buffers must stay valid until
 * the request finishes. */
nx_status nx_submit(nx_server* server, const nx_request* req, uint64_t* ticket);
/* nx_poll: NX_OK and the result once finished, NX_PENDING before. */
nx_status nx_poll(nx_server* server, uint64_t ticket, nx_result* result);
/* nx_wait: blocks until the request finishes or timeout_s passes
 * (NX_E_TIMEOUT; <= 0 waits without bound). */
nx_status nx_wait(nx_server* server, uint64_t ticket, nx_result* result, double timeout_s);
/* nx_cancel: withdraws a request.  A queued request is dropped at once; an
 * admitted one runs no further chunk, and its memory and request slot are
 * released once the chunk in flight has completed.  Its result status
 * becomes NX_E_CANCELED (nx_poll / nx_wait return it); its result buffers
 * are not written.  NX_E_STATE when it is too late: the request has finished
 * or its last chunk is already on the GPU (its result will arrive as
 * usual); NX_E_INVAL for an unknown ticket. */
nx_status nx_cancel(nx_server* server, uint64_t ticket);
nx_status nx_server_get_stats(nx_server* server, nx_server_stats* stats);
/* nx_server_destroy: finishes in-flight work, drops queued requests (their
 * status becomes NX_E_STATE) and releases everything. */
void nx_server_destroy(nx_server* server);

/* nx_rollout_noalloc: reset + rollout for callers that cannot allocate
 * device memory.  The paper has no counterpart; this exists for users of the
 * library whose process cannot call cudaMalloc: another runtime may already
 * hold nearly all of the device's memory in its own pool, or the calling loop
 * may not afford cudaMalloc's implicit device synchronisation.
 *
 * It does what nx_create(family, size, n_envs, seed, default options) +
 * nx_reset(NULL) + nx_rollout(n_steps, act_mode, d_actions_TN, traj) do, with
 * identical obs_sym, reward, terminated and truncated outputs, but allocates
 * nothing: the state, work list and request record live in one fixed device
 * array of NX_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds
 * until the process exits.  The caller passes the actions (device int8
 * [n_steps, n_envs], or NULL with NX_ACT_RANDOM) and the outputs (device,
 * [depth, n_envs, ...]).  Only obs_sym, reward, terminated and truncated are
 * written; every other nx_out pointer must be NULL (NX_E_INVAL otherwise).
 * Enqueued on cuda_stream, asynchronous.
 *
 * Limit: n_envs x (3 size^2 + 32) bytes plus a small work list must fit the
 * array (for example 3757 FourRooms-19x19 envs, or 4096 DoorKey-8x8 envs);
 * larger requests return NX_E_INVAL with the sizes in nx_last_error(NULL).
 * Every call looks up the array's device address in the current context
 * (cudaGetSymbolAddress, a host-side lookup); the first call on a device may
 * load the library's device code, so make that first call before any stream
 * capture.  Every call uses the same array and re-initialises what must
 * start from zero, so two calls that overlap on the GPU (different streams,
 * or different host threads) race and corrupt each other.  The sticky device
 * flags of nx_device_flags (an out-of-range action, a failed bounds check)
 * stay inside that array and no call reads them back: with NX_ACT_BUFFER,
 * pass actions in 0..6, since an out-of-range one runs as a no-op unseen. */
#define NX_NOALLOC_SCRATCH_BYTES (4u << 20)
nx_status nx_rollout_noalloc(int32_t family, int32_t size, int32_t n_envs, uint64_t seed, int32_t n_steps,
                             int32_t act_mode, const int8_t* d_actions_TN, const nx_out* traj, void* cuda_stream);

nx_status nx_profile_begin(nx_env* env);
nx_status nx_profile_end(nx_env* env, double* kernel_ms, int64_t* step_launches);
nx_status nx_launch_counts(const nx_env* env, int64_t* step_launches, int64_t* all_launches);
void nx_destroy(nx_env* env);
const char* nx_status_str(nx_status s);
const char* nx_last_error(const nx_env* env);

#ifdef __cplusplus
}
#endif
#endif
