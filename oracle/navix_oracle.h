/*
 * navix_oracle.h -- plain, single-threaded CPU oracle of the batched MiniGrid
 * step described in NAVIX (arXiv 2407.19396).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library
 * against an obviously-correct restatement of the paper's systems.  Only the
 * test-suite, the smoke check and the benchmark's CPU-baseline leg may load it;
 * the product library never links, loads or calls it, and it shares no source
 * with the CUDA side (its own Philox, its own layouts, rules, view and
 * visibility).  Compiled with -O2 -ffp-contract=off, no fast-math.
 *
 * What each function restates (paper sections/tables; the concrete readings
 * where the paper is silent are the project's documented readings R1-R18 and
 * L1-L5, restated next to the code that follows them):
 *   - the Intervention system (Table 3, Appendix A): rotate / forward /
 *     pickup / drop / toggle / done, with key-door colour matching (Table 2);
 *   - the Transition system (Table 3, Appendix A): Dynamic-Obstacles balls;
 *   - the rewards R1/R2/R3 of Table 8 and Table 5, terminations of Table 6,
 *     the optional non-Markovian MiniGrid reward of Eq. 1 (Section 3.2.1);
 *   - the timestep / reset padding / autoreset of Section 3.2.2 and Code 1;
 *   - the observations symbolic_first_person and rgb_first_person (Table 4);
 *   - the environment layouts of Table 8 (Empty, DoorKey, FourRooms, LavaGap,
 *     Dynamic-Obstacles).
 *
 * Parity pins: tests/test_oracle_*.py (Philox known-answer vectors, the
 * worked Empty-5x5 observation, hand sequences, BFS-optimal solves checked
 * against an independent rule model, brute-force visibility via an
 * independent rotate-then-occlude implementation, invariants).
 */
#ifndef NAVIX_ORACLE_H
#define NAVIX_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MIN_SIZE 5
#define ORC_MAX_SIZE 19
#define ORC_MAX_CELLS (ORC_MAX_SIZE * ORC_MAX_SIZE)
#define ORC_VIEW 7
#define ORC_OBS_BYTES (ORC_VIEW * ORC_VIEW * 3)
#define ORC_TILE 32
#define ORC_TILE_BYTES (ORC_TILE * ORC_TILE * 3)
#define ORC_RGB_BYTES (ORC_VIEW * ORC_TILE * ORC_VIEW * ORC_TILE * 3)
#define ORC_MAX_BALLS 4

/* families (variant: the number of rivers for the two crossing families) */
enum { ORC_EMPTY = 0, ORC_DOORKEY = 1, ORC_FOURROOMS = 2, ORC_LAVAGAP = 3, ORC_DYNOBS = 4, ORC_EMPTY_RANDOM = 5,
       ORC_LAVA_CROSSING = 6, ORC_SIMPLE_CROSSING = 7, ORC_GOTODOOR = 8, ORC_DISTSHIFT = 9,
       ORC_KEYCORRIDOR = 10 };
#define ORC_N_FAMILIES 11
#define ORC_NO_MISSION 255
/* actions */
enum { ORC_LEFT = 0, ORC_RIGHT = 1, ORC_FORWARD = 2, ORC_PICKUP = 3, ORC_DROP = 4, ORC_TOGGLE = 5, ORC_DONE = 6 };
/* entity codes */
enum { ORC_UNSEEN = 0, ORC_EMPTYCELL = 1, ORC_WALL = 2, ORC_FLOOR = 3, ORC_DOOR = 4, ORC_KEY = 5,
       ORC_BALL = 6, ORC_BOX = 7, ORC_GOAL = 8, ORC_LAVA = 9, ORC_AGENT = 10 };
/* colours */
enum { ORC_RED = 0, ORC_GREEN = 1, ORC_BLUE = 2, ORC_PURPLE = 3, ORC_YELLOW = 4, ORC_GREY = 5 };
/* door states */
enum { ORC_OPEN = 0, ORC_CLOSED = 1, ORC_LOCKED = 2 };
/* reward modes */
enum { ORC_REWARD_MARKOV = 0, ORC_REWARD_MINIGRID = 1 };

typedef struct orc_env {
    int32_t family, height, width, max_steps, n_balls, reward_mode, variant;
    float lava_reward;
    float action_cost, time_cost; /* Table 5's shaping terms (0 by default) */
    uint64_t seed;
    uint32_t env_index;
    uint32_t episode;
    int32_t t;                    /* steps since the last reset */
    int32_t ax, ay, dir;          /* agent position (x = column, y = row) and direction */
    int32_t carry_ent, carry_col; /* carry_ent == 0: nothing carried */
    int32_t done;                 /* previous call ended the episode: next call resets */
    int32_t mission;              /* GoToDoor: the colour of the target door; ORC_NO_MISSION otherwise */
    int32_t invalid_action;       /* sticky: an out-of-range action was seen */
    int32_t ball_x[ORC_MAX_BALLS], ball_y[ORC_MAX_BALLS];
    uint8_t ent[ORC_MAX_CELLS], col[ORC_MAX_CELLS], st[ORC_MAX_CELLS]; /* row-major y*W+x */
} orc_env;

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the bounded draw. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint32_t orc_bounded(uint32_t x, uint32_t n);
uint32_t orc_draw(uint64_t seed, uint32_t env_index, uint32_t episode, uint32_t step, uint32_t purpose,
                  uint32_t draw);

int32_t orc_default_max_steps(int32_t family, int32_t size);
int32_t orc_env_init(orc_env* e, int32_t family, int32_t size, int32_t max_steps, int32_t n_balls, uint64_t seed,
                     uint32_t env_index, int32_t reward_mode, float lava_reward, int32_t variant);
int32_t orc_max_variant(int32_t family, int32_t size);
/* action_cost / time_cost of Table 5 (both 0 after orc_env_init) */
void orc_set_costs(orc_env* e, float action_cost, float time_cost);
void orc_reset(orc_env* e, uint32_t episode);
int32_t orc_random_action(const orc_env* e, uint32_t gstep);
void orc_step(orc_env* e, int32_t action, float* reward, uint8_t* terminated, uint8_t* truncated);
void orc_obs_sym(const orc_env* e, uint8_t obs[ORC_OBS_BYTES]);
int32_t orc_tile_index(int32_t visible, int32_t agent_cell, int32_t ent, int32_t col, int32_t st);
/* Fully observable views (Table 4): symbolic [side][side][3] and categorical
 * [side][side], row-major over y then x, padded with zeros up to `side`
 * (>= the grid size); and categorical_first_person [7][7]. */
void orc_obs_full(const orc_env* e, uint8_t* full, int32_t side);
void orc_obs_cat(const orc_env* e, uint8_t* cat, int32_t side);
void orc_obs_cat_fp(const orc_env* e, uint8_t cat[ORC_VIEW * ORC_VIEW]);
/* rgb (Table 4): the whole grid as 32-px sprites, [32 side][32 side][3]; a
 * cell (e, c, s) uses tile 1 + 18 e + 3 c + s, the agent's cell tile
 * 397 + direction, cells beyond the grid tile 0. */
void orc_obs_rgb_full(const orc_env* e, const uint8_t* atlas, uint8_t* img, int32_t side);
void orc_obs_rgb(const orc_env* e, const uint8_t* atlas, uint8_t* img);

/* hand-built states for the worked sequences */
void orc_set_cell(orc_env* e, int32_t x, int32_t y, int32_t ent, int32_t col, int32_t st);
void orc_set_agent(orc_env* e, int32_t x, int32_t y, int32_t dir, int32_t carry_ent, int32_t carry_col);

/* Batch convenience used by the tests and the CPU baseline: n environments,
 * stepped one after another in index order, all with the same seed and
 * global env indices 0..n-1.  Output arrays are [n, ...]; any may be NULL. */
/* A policy for the fused policy + environment rollout (the PPO rollout
 * pattern of Section 4's batch-mode experiment, reading P1): an integer MLP
 * from the categorical first-person view (49 entity codes) to one logit per
 * action.  For each hidden unit j:
 *   h1[j] = clamp((sum_k w1[j][k] x[k] + b1[j]) >> shift1, 0, 255)
 *   h2[j] = clamp((sum_i w2[j][i] h1[i] + b2[j]) >> shift2, 0, 255)
 *   z[a]  = sum_i w3[a][i] h2[i] + b3[a]
 * (>> is the floor of division by 2^shift), the greedy action is the first
 * index of the largest z[a] over the family's actions, and with probability
 * epsilon / 2^32 (an exploration draw below epsilon) the action is the
 * uniform random action instead.  Env e uses weight set e / envs_per_agent. */
#define ORC_HIDDEN 64
#define ORC_POLICY_IN 49
typedef struct {
    int32_t n_agents, envs_per_agent;
    const int8_t* w1;  /* [n_agents][64][49] */
    const int32_t* b1; /* [n_agents][64] */
    const int8_t* w2;  /* [n_agents][64][64] */
    const int32_t* b2; /* [n_agents][64] */
    const int8_t* w3;  /* [n_agents][7][64] */
    const int32_t* b3; /* [n_agents][7] */
    int32_t shift1, shift2;
    uint32_t epsilon;
} orc_policy;
/* the greedy action of weight set `agent` for a categorical view (first max) */
int32_t orc_policy_greedy(const orc_policy* p, int32_t agent, const uint8_t* cat_fp, int32_t n_act);
/* the action the policy takes in env e at global step gstep */
int32_t orc_policy_action(const orc_policy* p, const orc_env* e, uint32_t gstep);

typedef struct orc_batch orc_batch;
orc_batch* orc_batch_create(int32_t n, const int32_t* family, const int32_t* size, const int32_t* max_steps,
                            const int32_t* variant, int32_t n_balls, uint64_t seed, uint32_t env_index_base,
                            int32_t reward_mode, float lava_reward);
/* as above, with an explicit global env index per env (a sample of a larger batch) */
orc_batch* orc_batch_create_indexed(int32_t n, const int32_t* family, const int32_t* size, const int32_t* max_steps,
                                    const int32_t* variant, int32_t n_balls, uint64_t seed, const uint32_t* env_index,
                                    int32_t reward_mode, float lava_reward);
void orc_batch_destroy(orc_batch* b);
void orc_batch_set_costs(orc_batch* b, float action_cost, float time_cost);
orc_env* orc_batch_env(orc_batch* b, int32_t i);
void orc_batch_reset(orc_batch* b, uint8_t* obs_sym, uint8_t* obs_rgb, const uint8_t* atlas, float* reward,
                     uint8_t* terminated, uint8_t* truncated);
/* actions == NULL: random actions from the counter hash at the batch's global
 * step counter (which every call advances by one). */
void orc_batch_step(orc_batch* b, const int8_t* actions, uint8_t* obs_sym, uint8_t* obs_rgb, const uint8_t* atlas,
                    float* reward, uint8_t* terminated, uint8_t* truncated);
/* T steps in a row; outputs are [T, n, ...] (any may be NULL) */
void orc_batch_rollout(orc_batch* b, int32_t T, const int8_t* actions_TN, uint8_t* obs_sym, uint8_t* obs_rgb,
                       const uint8_t* atlas, float* reward, uint8_t* terminated, uint8_t* truncated);
uint32_t orc_batch_gstep(const orc_batch* b);
/* T steps with the policy choosing every env's action from its current
 * categorical view; actions_out [T, n] (may be NULL) receives the actions. */
void orc_batch_rollout_policy(orc_batch* b, int32_t T, const orc_policy* p, int8_t* actions_out, uint8_t* obs_sym,
                              float* reward, uint8_t* terminated, uint8_t* truncated);
/* the current fully observable views of every env ([n, side, side, 3],
 * [n, side, side], [n, 7, 7]; any may be NULL) */
void orc_batch_obs_full(orc_batch* b, uint8_t* full, uint8_t* cat, uint8_t* cat_fp, int32_t side);
void orc_batch_obs_rgb_full(orc_batch* b, const uint8_t* atlas, uint8_t* img, int32_t side);

#ifdef __cplusplus
}
#endif
#endif
