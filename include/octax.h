/*
 * liboctax: data-parallel CHIP-8 environment step on one GB300 (sm_103a).
 *
 * C-ABI boundary of the vectorised environment step described by the Octax
 * paper (arXiv 2510.01764): many independent CHIP-8 emulator instances, each
 * stepping with fetch/decode/execute of the 35 instructions (§3.2
 * "Fetch-decode-execute cycle", App. B), an XOR sprite blit with VF collision
 * into a 64x32 1-bit display (App. B "Sprite Drawing"), 60 Hz delay/sound
 * timers, K instructions per frame with frame skip and a stacked observation
 * (§3.2 "Environment integration", §4.2), and reward/termination read from
 * game registers or memory with automatic reset (§3.3). Games may instead be
 * Super-CHIP programs, the 128x64 extension named in §5 (OCTAX_VARIANT_SCHIP,
 * one variant per environment): lores/hires modes, 16x16 sprites, scrolls,
 * 8x10 glyphs and flag registers, with uint8 [S][64][128] observations.
 *
 * Conventions (every entry point):
 *  - Plain pointers and sizes only. "_dev" pointers are CUDA device memory
 *    owned by the caller (e.g. a torch tensor's data_ptr()); "_host" pointers
 *    are host memory owned by the caller (pinned memory copies fastest).
 *    The library owns the emulator state and the ROM images; `rom` bytes are
 *    copied at creation.
 *  - Return value: OCTAX_OK (0) or a negative OCTAX_E* code; the message of
 *    the last failure on the calling thread is octax_last_error().
 *  - Work is enqueued on the environment's CUDA stream and the call returns
 *    without waiting, except where a function says it is synchronous.
 *  - Device-side faults never trap: stack over/underflow, invalid opcodes and
 *    out-of-range action indices set per-instance status bits.
 *  - Results are bit-exact and independent of launch configuration, batch
 *    composition and instance placement.
 */
#ifndef OCTAX_H
#define OCTAX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes --------------------------------------------------------- */
#define OCTAX_OK 0
#define OCTAX_EINVAL (-1)   /* bad argument: sizes, descriptor fields, null pointer */
#define OCTAX_ENOMEM (-2)   /* device or host allocation failed / over budget       */
#define OCTAX_ECUDA (-3)    /* a CUDA runtime call failed (message has the detail)  */
#define OCTAX_ETIMEOUT (-4) /* octax_sync / server wait deadline passed             */
#define OCTAX_ENOTFOUND (-5) /* unknown request id                                 */

/* ---- quirk bits (one env-wide bit set; 0 = the classic set) -------------- */
#define OCTAX_QUIRK_SHIFT_USES_VY 0x01u   /* 8XY6/8XYE shift VY into VX          */
#define OCTAX_QUIRK_LOADSTORE_INC_I 0x02u /* FX55/FX65 leave I = I + X + 1       */
#define OCTAX_QUIRK_LOGIC_RESETS_VF 0x04u /* 8XY1/8XY2/8XY3 set VF = 0           */
#define OCTAX_QUIRK_JUMP_VX 0x08u         /* BXNN jumps to XNN + VX              */
#define OCTAX_QUIRK_WRAP_SPRITES 0x10u    /* DXYN wraps at the display edges     */
#define OCTAX_QUIRK_FX1E_VF 0x20u         /* FX1E sets VF = (I + VX > 0xFFF)     */

/* ---- per-instance status bits (sticky since creation) -------------------- */
#define OCTAX_STATUS_BAD_OP 0x01u      /* an undefined opcode was executed (no-op) */
#define OCTAX_STATUS_STACK_FAULT 0x02u /* CALL on a full / RET on an empty stack   */
#define OCTAX_STATUS_BAD_ACTION 0x04u  /* action index > n_actions (no key held)   */
#define OCTAX_STATUS_EXIT 0x08u        /* SCHIP 00FD executed (the program halts)  */

/* ---- instruction-set variant (octax_game.variant) --------------------------- */
#define OCTAX_VARIANT_CHIP8 0u /* 64x32 display, observation frames of 32 x 64 bytes       */
#define OCTAX_VARIANT_SCHIP 1u /* 128x64 buffer (lores: 64x32 grid of 2x2 blocks), frames of
                                  64 x 128 bytes; adds 00CN 00FB 00FC 00FD 00FE 00FF, DXY0
                                  (16x16), FX30 (8x10 glyphs at 0x0A0), FX75 / FX85 (16
                                  flag bytes, cleared at reset). Every episode starts in
                                  lores; scroll distances count pixels of the current
                                  mode; mode switches keep the buffer; 00FD re-executes
                                  itself and sets OCTAX_STATUS_EXIT; VF = any collision. */

/* ---- reward / termination descriptor (§3.3 score_fn / terminated_fn) ----- */
enum { OCTAX_SRC_REG = 0, OCTAX_SRC_MEM = 1 };
enum {
  OCTAX_X_RAW = 0,                 /* v                                  */
  OCTAX_X_NEG = 1,                 /* -v                                 */
  OCTAX_X_DEC_TENS = 2,            /* v / 10                             */
  OCTAX_X_DEC_ONES = 3,            /* v % 10                             */
  OCTAX_X_DEC_TENS_MINUS_ONES = 4, /* v/10 - v%10 (Pong, §3.3)          */
  OCTAX_X_NIB_HI_MINUS_LO = 5,     /* (v >> 4) - (v & 15)               */
  OCTAX_X_ZERO_IF_GT = 6           /* v > arg ? 0 : v (App. C)          */
};
enum { OCTAX_CMP_EQ = 0, OCTAX_CMP_NE, OCTAX_CMP_GE, OCTAX_CMP_GT, OCTAX_CMP_LE, OCTAX_CMP_LT };

typedef struct {
  uint8_t src;   /* OCTAX_SRC_REG: V[idx & 15]; OCTAX_SRC_MEM: RAM[idx & 0xFFF] */
  uint8_t xform; /* OCTAX_X_*                                                  */
  uint16_t idx;
  int32_t arg;   /* threshold of OCTAX_X_ZERO_IF_GT                            */
} octax_term;    /* 8 bytes */

typedef struct {
  octax_term lhs;
  uint8_t cmp;   /* OCTAX_CMP_*: lhs <cmp> rhs */
  uint8_t pad[3];
  int32_t rhs;
} octax_clause;  /* 16 bytes */

/* One game (§3.2-§3.3): ROM, timing, action set, reward and termination. */
typedef struct {
  const uint8_t *rom;        /* host pointer, 1..3584 bytes, loaded at 0x200; copied */
  uint32_t rom_len;
  uint8_t instr_per_frame;   /* K >= 1 (the paper's ~700 Hz is ~11.7 per frame)       */
  uint8_t frameskip;         /* frames per env step >= 1 (paper default 4)            */
  uint8_t stack_frames;      /* frames in the observation, 1..frameskip; same for all
                                games of one environment                             */
  uint8_t n_actions;         /* 0..16; action index n_actions means "no key"          */
  uint8_t action_set[16];    /* action index -> CHIP-8 key (0..15)                    */
  uint8_t n_score_terms;     /* 0..4: score = sum of terms                            */
  uint8_t n_term_clauses;    /* 0..4: terminated = OR of clauses (0 = never)          */
  uint8_t variant;           /* OCTAX_VARIANT_*; the same for all games of one
                                environment (or server)                              */
  uint8_t pad;
  octax_term score[4];
  octax_clause term[4];
  uint32_t max_episode_steps; /* truncation after this many steps; 0 = none           */
  uint32_t startup_instrs;    /* instructions run at every reset with no key held,
                                 0..2^20                                             */
  uint32_t sticky_threshold;  /* sticky actions (§3.2 wrappers): at every env step the
                                 previous step's action index is applied instead of
                                 the caller's when Philox4x32-10 word 0 at counter
                                 (uid, env_steps, 0, 2) is below this; probability
                                 p -> round(p * 2^32); 0 = off. A new episode's
                                 previous action is the no-op (index n_actions). */
  uint32_t max_noops;         /* no-op reset (§3.2 wrappers): after the startup
                                 instructions every reset runs (word 0 at counter
                                 (uid, env_steps, 0, 3)) mod (max_noops + 1) env
                                 steps with no key held and nothing observed;
                                 0..255, 0 = off                                    */
} octax_game;                 /* 152 bytes */

/* Canonical state of one instance: the unit of comparison and checkpointing.
 * RAM is the full 4 KB as the program sees it (font, ROM and all writes). */
typedef struct {
  uint8_t V[16];
  uint16_t I, PC;
  uint8_t SP;                /* occupied call-stack entries, 0..16 */
  uint8_t DT, ST, status;
  uint16_t stack[16];
  uint64_t display[64][2];   /* bit (x mod 64) of display[y][x / 64] = pixel (x, y);
                                CHIP-8 uses rows 0-31, word 0 (other words are 0) */
  uint8_t ram[4096];
  uint32_t episode_steps;    /* steps since the last reset */
  uint32_t env_steps;        /* steps since creation (random-number counter) */
  uint8_t last_action;       /* action index applied at the previous step (sticky
                                actions); n_actions after a reset */
  uint8_t hires;             /* SCHIP: 1 in 128x64 mode */
  uint8_t pad[6];
  uint8_t rpl[16];           /* SCHIP flag registers (FX75 / FX85) */
} octax_state_record;        /* 5208 bytes. octax_state_hash is FNV-1a 64 over, in
                                order and little-endian: V, I, PC, SP, DT, ST, status,
                                stack, the display (CHIP-8: display[0..31][0]; SCHIP:
                                all [64][2] row-major), ram, episode_steps, env_steps,
                                last_action, and for SCHIP hires and rpl            */

/* Launch configuration (chosen by octax_autotune or set by hand). A CTA of
 * `block` emulator threads runs block/32 * inst_per_warp instances of one
 * game; with writer_warps > 0 it also has that many warps that only write
 * observations (block/32 * inst_per_warp / writer_warps must be 8, 16 or 32;
 * CHIP-8 environments only). */
typedef struct {
  int32_t block;             /* emulator threads per CTA: 32, 64, 128 or 256    */
  int32_t inst_per_warp;     /* instances emulated per warp: 1..32                */
  int32_t steps_per_launch;  /* octax_step_n: env steps per kernel launch 1..256 */
  int32_t persistent;        /* 1: resident CTAs pull instance groups off a queue */
  int32_t use_graph;         /* 1: octax_step_n replays a captured CUDA graph     */
  int32_t writer_warps;      /* 0, 1, 2, 4 or 8 observation-writer warps         */
  int32_t balance;           /* 1: spread the instances evenly over a whole number
                                of waves of resident CTAs (every SM gets the same
                                number of CTAs); 0: full CTAs, ragged last one   */
} octax_launch;

typedef struct octax_env octax_env;

/* Create n_envs instances over n_games games and reset them all (§3.2 "ROM
 * loading and initialization"). game_of_env[i] (host, nullable = all 0) picks
 * instance i's game; uid_of_env[i] (host, nullable = i) is its random-number
 * identity, so an instance's trajectory depends only on (seed, uid, actions).
 * cuda_stream: a cudaStream_t (NULL = legacy default stream). Synchronous.
 * EINVAL: n_games < 1, n_envs < 1, a descriptor field out of range, unknown
 * quirk bits, stack_frames differing between games. */
int octax_create(const octax_game *games, int n_games, const uint16_t *game_of_env,
                 const uint32_t *uid_of_env, int64_t n_envs, uint32_t quirks,
                 uint64_t seed, void *cuda_stream, octax_env **out);

/* Reset the instances with mask_dev[i] != 0 (mask_dev NULL = all) and write
 * their observation. The reset is the paper's episode start (§3.2 "ROM
 * loading and initialization": memory image, registers, PC = 0x200) followed
 * by the game's startup instructions (§3.3 "Initialization handling"); the
 * reward baseline is the score after them. The observation (the reset
 * display in every stack slot) goes to obs_dev[i][stack_frames][H][W] (uint8 0/1; NULL = no write). H x W is 32 x 64
 * for CHIP-8 and 64 x 128 for SCHIP environments. */
int octax_reset(octax_env *env, const uint8_t *mask_dev, uint8_t *obs_dev);

/* One environment step for every instance (§3.2, §4.2).
 * actions_dev: uint8 [n_envs], index into the game's action_set.
 * obs_dev: uint8 [n_envs][stack_frames][H][W], the last stack_frames frames
 *   of the step, oldest first; for a done instance the reset display.
 * reward_dev: float32 [n_envs], score after minus score before the step.
 * done_dev: uint8 [n_envs], terminated or truncated; done instances are reset. */
int octax_step(octax_env *env, const uint8_t *actions_dev, uint8_t *obs_dev,
               float *reward_dev, uint8_t *done_dev);

/* n_steps steps in as few launches as the launch configuration allows. The
 * paper steps one env step per call (§3.2, §4.2); this batched form is the
 * "adaptive batching" that §5 names as future work for the synchronisation
 * cost of uneven instruction counts: many steps, games with different
 * instructions per frame and uneven episodes in one persistent or
 * graph-replayed launch.
 * (steps_per_launch per launch, CUDA-graph replay, persistent scheduling).
 * actions_dev [n_steps][n_envs]; obs_dev [n_steps][n_envs][S][H][W];
 * reward_dev, done_dev [n_steps][n_envs]. Same results as n_steps octax_step. */
int octax_step_n(octax_env *env, int n_steps, const uint8_t *actions_dev, uint8_t *obs_dev,
                 float *reward_dev, uint8_t *done_dev);

/* octax_step_n writing packed observations (the paper's observation is a
 * boolean frame stack, §3.2 "4-frame stacking", §4.1), one bit per pixel instead of one
 * byte (8x fewer observation bytes): obs_words_dev is uint64 [n_steps][n_envs]
 * [S][W], 16-byte aligned, with W = 32 for CHIP-8 (word y = row y, bit x =
 * pixel x) and 128 for SCHIP (word 2y + h = pixels 64h..64h+63 of row y, bit x
 * = pixel 64h + x). The frames hold the same pixels as octax_step_n's; rewards,
 * done flags and state are identical. Writer warps are not used for these
 * calls. */
int octax_step_n_packed(octax_env *env, int n_steps, const uint8_t *actions_dev, uint64_t *obs_words_dev,
                        float *reward_dev, uint8_t *done_dev);

/* octax_step (§3.2) with host buffers, synchronous. Page-locked (pinned) buffers are
 * read and written by the kernel directly through their device mapping;
 * pageable buffers go through device staging buffers and copies. */
int octax_step_host(octax_env *env, const uint8_t *actions_host, uint8_t *obs_host,
                    float *reward_host, uint8_t *done_host);

/* octax_step_host writing packed frames (layout of octax_step_n_packed) into
 * obs_words_host [n_envs][S][W]: 8x fewer bytes over the host link. */
int octax_step_host_packed(octax_env *env, const uint8_t *actions_host, uint64_t *obs_words_host,
                           float *reward_host, uint8_t *done_host);

/* FNV-1a 64-bit hash of each instance's canonical record (octax_state_record
 * bytes in field order, little-endian) into hash_dev [n_envs]. The paper
 * defines no counterpart: this is the parity check against the CPU oracle.
 * Asynchronous on the environment's stream; EINVAL for a NULL argument. */
int octax_state_hash(octax_env *env, uint64_t *hash_dev);

/* Copy the canonical records of instances [first, first+count) to host
 * memory. The paper defines no counterpart (state comparison with the
 * oracle, checkpoints). Synchronous. EINVAL if the range is outside
 * [0, n_envs). */
int octax_get_state(octax_env *env, int64_t first, int64_t count, octax_state_record *out_host);

/* Overwrite instances [first, first+count) from records (checkpoint resume;
 * the paper defines no counterpart).
 * Synchronous. EINVAL if the range is outside [0, n_envs) or SP > 16. */
int octax_set_state(octax_env *env, int64_t first, int64_t count,
                    const octax_state_record *in_host);

/* Wait until all enqueued work finished (the paper defines no counterpart:
 * its JAX calls block implicitly); OCTAX_ETIMEOUT after timeout_ms
 * (negative = no limit). OCTAX_ECUDA if a kernel reported an internal
 * hand-over timeout since the last octax_sync: the outputs of the calls
 * since then are incomplete and the state of the instances in the failed
 * CTAs is left as it was before the failed launch. The report clears the
 * flag, so the environment stays usable. */
int octax_sync(octax_env *env, int timeout_ms);

/* Diagnostic (the paper defines no counterpart) for the failure path of the warp-specialised kernel
 * (writer_warps > 0): while `on` is nonzero its writer warps skip their
 * shared-memory hand-over, so the emulator warps' bounded waits (at most
 * about one second each) run out, the kernel records the failure and
 * returns, and octax_sync reports OCTAX_ECUDA. No other kernel is affected.
 * Drops the cached CUDA graphs so that the next launches see the switch. */
int octax_debug_stall_writers(octax_env *env, int on);

/* Read / set the launch configuration (the paper defines no counterpart:
 * XLA picks its own launches). EINVAL for unsupported values. */
int octax_get_launch(const octax_env *env, octax_launch *out);
int octax_set_launch(octax_env *env, const octax_launch *cfg);

/* Autotuner for the batched step (part of §5's adaptive batching; the paper
 * defines no tuner). Times candidate launch configurations (CTA size, instances per warp, steps
 * per launch from 1 to 256 and n_steps itself, persistence, writer warps) for
 * octax_step_n calls of n_steps steps, starting
 * from the current state, then restore that state: results are unaffected.
 * actions_dev [n_steps][n_envs] (nullable: pseudo-random indices 0..4) should
 * be representative, since divergence depends on them. Keeps the fastest
 * configuration. Synchronous. best_ms_out (nullable) receives its time. */
int octax_autotune(octax_env *env, int n_steps, const uint8_t *actions_dev, float *best_ms_out);

/* Accessors (the paper defines no counterparts); -1 / 0 for a NULL env. */
int64_t octax_num_envs(const octax_env *env);
int octax_stack_frames(const octax_env *env);
/* OCTAX_VARIANT_CHIP8 or OCTAX_VARIANT_SCHIP. */
int octax_variant(const octax_env *env);
/* Device bytes owned by the environment. */
size_t octax_device_bytes(const octax_env *env);
/* Free the environment's device memory once its queued work has finished
 * (the paper defines no counterpart). NULL is a no-op. */
void octax_destroy(octax_env *env);

/* ---- serving: continuous batching of step requests ------------------------
 * The paper defines no server; its consumers are training loops that step
 * batches of environments (§4.1), and the request loop here batches such
 * step requests as they arrive. A server keeps a pool of resident emulator slots sized by a device-memory
 * budget and runs its own thread and CUDA stream. Each request asks for
 * n_envs fresh instances of one game (reset with its own seed; instance i has
 * random-number identity i) stepped n_steps times with the given actions.
 * Queued requests are admitted first-in first-out as slots free up; every
 * scheduling tick launches one step kernel over all admitted requests, each
 * at its own step, advancing them all by the fewest steps any of them has
 * left (at least one), so requests that arrive while others run join the
 * next tick, and a request that runs alone takes one launch. Results are
 * identical to running the request alone (octax_create + octax_step with the
 * same seed). */
typedef struct octax_server octax_server;

typedef struct {
  int64_t memory_budget_bytes; /* device bytes for resident instance state; the
                                  slot pool holds budget / 4,476 instances
                                  (4,468 B of state and 8 B of per-step
                                  buffers each; Super-CHIP: budget / 5,244)   */
  int32_t block;               /* threads per CTA: 32, 64, 128, 256 (0 = 64)    */
  int32_t inst_per_warp;       /* 1, 2, 4, 8, 16, 32 (0 = 8)                    */
  int32_t max_inflight_ticks;  /* batched launches enqueued ahead, 1..8 (0 = 2) */
  int32_t reserved;
} octax_server_config;

typedef struct {
  uint16_t game;               /* index into the server's games               */
  uint16_t pad;
  uint32_t n_envs;             /* 1..4096                                     */
  uint32_t n_steps;            /* 1..8                                        */
  uint32_t pad2;
  uint64_t seed;               /* Philox key of this request's instances     */
  const uint8_t *actions_host; /* [n_steps][n_envs] action indices, copied    */
  uint8_t *obs_dev;            /* [n_steps][n_envs][S][H][W], 16-byte aligned */
  float *reward_dev;           /* [n_steps][n_envs]                           */
  uint8_t *done_dev;           /* [n_steps][n_envs]                           */
} octax_request;               /* the caller keeps the device buffers alive until done */

typedef struct {
  int32_t state;               /* 0 queued, 1 running, 2 done                 */
  int32_t pad;
  int64_t submit_ns, admit_ns, done_ns; /* steady-clock timestamps (ns)       */
} octax_request_info;

typedef struct {
  int64_t submitted, completed, env_steps, ticks;
  int64_t peak_active_envs, peak_active_requests;
  int64_t slots_capacity, slots_in_use, queued;
} octax_server_stats;

/* Start a server over n_games games (same descriptor rules as octax_create).
 * EINVAL: bad descriptors / config; ENOMEM: the budget cannot be allocated. */
int octax_server_create(const octax_game *games, int n_games, uint32_t quirks,
                        const octax_server_config *cfg, octax_server **out);
/* Queue a request (thread-safe, returns at once). EINVAL: bad fields;
 * ENOMEM: n_envs exceeds the whole slot pool. */
int octax_server_submit(octax_server *s, const octax_request *req, uint64_t *id_out);
/* Queue n requests under one lock (all or none: EINVAL / ENOMEM as for
 * octax_server_submit, nothing queued). ids_out [n] receives their ids in
 * order. For load generators and clients that produce many small requests,
 * whose one-by-one submission would cost more host time than their GPU work.
 * The paper defines no counterpart. */
int octax_server_submit_batch(octax_server *s, const octax_request *reqs, int n, uint64_t *ids_out);
/* Wait until request id is done (its outputs are then complete in device
 * memory). timeout_ms < 0 waits without limit; ETIMEOUT, ENOTFOUND. */
int octax_server_wait(octax_server *s, uint64_t id, int timeout_ms, octax_request_info *info_out);
/* Wait until all n requests ids [n] are done (timeout_ms for the whole wait,
 * < 0 = no limit), copy their infos into infos [n] (nullable) and, if release
 * is nonzero, forget them as octax_server_release does. ETIMEOUT, ENOTFOUND
 * (nothing released). The paper defines no counterpart. */
int octax_server_wait_batch(octax_server *s, const uint64_t *ids, int n, int timeout_ms, octax_request_info *infos,
                            int release);
int octax_server_query(octax_server *s, uint64_t id, octax_request_info *info_out);
/* Forget a finished request's bookkeeping. EINVAL if it is not done. */
int octax_server_release(octax_server *s, uint64_t id);
int octax_server_get_stats(octax_server *s, octax_server_stats *out);
/* Finish enqueued work, stop the thread, free the pool. */
void octax_server_destroy(octax_server *s);

/* ---- no-allocation entry point ---------------------------------------------
 * The paper has no counterpart to this call; it exists for callers that may
 * not allocate device memory: code running inside another framework's
 * memory pool or a pre-reserved arena, plugins whose host forbids
 * allocation after start-up, and real-time loops where an allocation (which
 * can synchronise the device) would break the timing budget.
 * Runs n_envs fresh instances of one game (reset with `seed`; instance i has
 * random-number identity i) for n_steps steps, exactly what octax_create +
 * octax_step_n compute, but with every piece of scratch state in one
 * library-owned static device array of fixed size, so the call allocates
 * nothing. Inputs and outputs are the caller's device buffers, as in
 * octax_step_n: actions_dev [n_steps][n_envs]; obs_dev
 * [n_steps][n_envs][stack_frames][32][64] (16-byte aligned); reward_dev and
 * done_dev [n_steps][n_envs]. Asynchronous on cuda_stream (NULL = legacy
 * default stream).
 * Limits: 1 <= n_envs <= 1024 (EINVAL beyond); CHIP-8 games only (EINVAL
 * for OCTAX_VARIANT_SCHIP); every device that loads the
 * library holds the array (about 4.6 MB) until the process exits.
 * The first call on a device looks up the array's device address, so make it
 * before any stream capture. The address is kept for the life of the
 * process: do not call this entry point again on a device after
 * cudaDeviceReset on it (the cached address belongs to the ended context). Every call reuses the same array: calls whose
 * work overlaps on the GPU (other streams, other threads) race with each
 * other and must be serialised by the caller. */
int octax_rollout_static(const octax_game *game, int64_t n_envs, uint32_t quirks, uint64_t seed,
                         int n_steps, const uint8_t *actions_dev, uint8_t *obs_dev,
                         float *reward_dev, uint8_t *done_dev, void *cuda_stream);

/* ---- the policy network and the on-device rollout -------------------------
 * The actor-critic network that consumes the observation stack (§4.1,
 * "Network architecture"): three convolutions (32 filters, kernel (8,4),
 * stride (4,2); 64 filters, 4, 2; 64 filters, 3, 1) with ReLU over the
 * 4-frame stack in the (frame, x, y) = (4, 64, 32) orientation, VALID
 * padding (64 x 32 -> 15 x 15 -> 6 x 6 -> 4 x 4), the 1,024 features
 * flattened in (channel, x, y) order, then an actor head (256 ReLU units ->
 * n_logits logits) and a critic head (256 ReLU units -> one value). The
 * convolutions and hidden layers run on the tensor cores with bfloat16
 * weights and activations and fp32 accumulation; the output layers and the
 * action draw run in fp32. */
typedef struct octax_policy octax_policy;

/* Parameters, host float32 arrays in these layouts (copied at creation):
 * w1 [32][4][8][4] (out, frame, kx, ky), b1 [32]; w2 [64][32][4][4], b2 [64];
 * w3 [64][64][3][3], b3 [64]; wa1, wc1 [256][1024] (input index = channel * 16
 * + x * 4 + y), ba1, bc1 [256]; wa2 [n_logits][256], ba2 [n_logits];
 * wc2 [256], bc2 [1]. n_logits = the game's n_actions + 1 (its action
 * indices, the no-op last), 1..17. */
typedef struct {
  const float *w1, *b1, *w2, *b2, *w3, *b3;
  const float *wa1, *ba1, *wa2, *ba2;
  const float *wc1, *bc1, *wc2, *bc2;
  int32_t n_logits;
} octax_policy_params;

/* Create a policy on `device` for batches of up to max_envs instances (its
 * device buffers: packed weights 1.2 MB, features 2 KB and a two-slot packed
 * observation ring 2 KB per instance). cuda_stream: the stream of
 * octax_policy_forward calls (NULL = a stream of its own). Synchronous.
 * EINVAL: a NULL array, n_logits outside 1..17, max_envs outside 1..2^31. */
int octax_policy_create(const octax_policy_params *params, int64_t max_envs, int device, void *cuda_stream,
                        octax_policy **out);

/* The network on n_envs packed observation stacks obs_words_dev [n][4][32]
 * (the layout of octax_step_n_packed: word y of frame f = row y, bit x =
 * pixel x; 16-byte aligned). Outputs (each nullable): logits_dev
 * [n][n_logits] and value_dev [n] (fp32), actions_dev [n]: an action index
 * drawn from softmax(logits) by inverse CDF, with u = (w >> 8) * 2^-24 for
 * the Philox4x32-10 word w at key = seed (low word first) and counter =
 * (instance index, step, 0, 0). Asynchronous on the policy's stream.
 * EINVAL: n_envs outside 1..max_envs, unaligned input. */
int octax_policy_forward(octax_policy *policy, int64_t n_envs, const uint64_t *obs_words_dev, uint64_t seed,
                         uint32_t step, float *logits_dev, float *value_dev, uint8_t *actions_dev);

/* The same on uint8 observation stacks obs_dev [n][4][32][64] (the layout
 * of octax_step_n; a nonzero byte is a lit pixel). */
int octax_policy_forward_u8(octax_policy *policy, int64_t n_envs, const uint8_t *obs_dev, uint64_t seed,
                            uint32_t step, float *logits_dev, float *value_dev, uint8_t *actions_dev);

/* On-device rollout of n_steps steps in which the policy picks every action
 * (the acting loop of the paper's PPO training, §4.1): for step k the
 * network runs on the current observation and draws actions (counter step =
 * step0 + k), then the environment steps with them. Observations pass
 * between the two as packed frames through the policy's two-slot ring
 * (1 KB per instance; no uint8 frames are written). obs_words_dev
 * [n][4][32] holds the current observation on entry (from octax_reset
 * packed by the caller, or a previous rollout) and the observation after
 * the last step on return. Outputs per step: actions_dev [n_steps][n],
 * logits_dev [n_steps][n][n_logits] (nullable), value_dev [n_steps][n],
 * reward_dev and done_dev [n_steps][n] as octax_step_n. Asynchronous on the
 * environment's stream. EINVAL: not a CHIP-8 environment with 4 stacked
 * frames, more instances than max_envs, another device. */
int octax_rollout_policy(octax_env *env, octax_policy *policy, int n_steps, uint64_t seed, uint32_t step0,
                         uint64_t *obs_words_dev, uint8_t *actions_dev, float *logits_dev, float *value_dev,
                         float *reward_dev, uint8_t *done_dev);

/* Wait for the policy's stream and the device; OCTAX_ECUDA (once) if a
 * policy kernel gave up one of its bounded waits (its outputs are then
 * incomplete). The paper defines no counterpart. */
int octax_policy_sync(octax_policy *policy);
/* Diagnostic for the policy kernels' failure path (the paper defines no
 * counterpart): while `on` is nonzero the conv kernel skips the completion
 * signal of its first MMA group, so that wait runs out after about one
 * second in every CTA; the kernel records the failure and returns, and the
 * next octax_policy_sync reports OCTAX_ECUDA. No other work is affected. */
int octax_policy_debug_stall(octax_policy *policy, int on);
void octax_policy_destroy(octax_policy *policy);

/* Message of the last failed call on this thread ("" if none). The paper
 * defines no counterpart. */
const char *octax_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
