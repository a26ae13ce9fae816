/*
 * Octax CHIP-8 environment oracle: plain, slow, single-instance CPU reference.
 *
 * TEST INFRASTRUCTURE ONLY. The test-suite, the smoke check and the benchmark's
 * CPU-baseline leg are the only users of this code; the product library never
 * links, loads or calls it, and it shares no code, header, table or constant
 * with the CUDA implementation.
 *
 * Source of truth: the Octax paper (arXiv 2510.01764).
 *   §3.2  ROM loading at 0x200, font at 0x50, V0-VF, I, PC, 64x32 display;
 *         fetch/decode/execute; K instructions per step; frame skip; 4-frame
 *         observation stack; action set + no-op; 60 Hz timers; startup
 *         instructions; RND makes games stochastic.
 *   §3.3  score_fn / terminated_fn read game registers (compound OR clauses).
 *   §4.2  default frame skip of 4 frames per environment step.
 *   App. B  4 KB memory, 16 8-bit registers with VF as flag register, 64x32
 *         XOR display, 16-key keypad, delay/sound timers, DXYN / EX9E / EXA1 /
 *         FX33 / FX55 / FX65, font at 0x050-0x09F.
 *   App. C  per-game score and termination expressions.
 * The paper names the 35-instruction set without spelling out each opcode; the
 * semantics here are the classic CHIP-8 definition. Every point the paper leaves
 * open is marked READING in octax_oracle.c.
 *
 * §5 (future work) names the Super-CHIP8 extension: a 128x64 display and the
 * instruction set extended for HP48 calculators. The paper defines neither, so
 * the SCHIP variant here follows the published Super-CHIP 1.1 instruction
 * list; every point where interpreters differ is marked READING.
 *
 * Parity unpinned: the 4x5 font glyph bytes (the paper fixes only their address
 * range 0x050-0x09F, App. B "Font System") and the 8x10 SCHIP glyphs (not in
 * the paper at all).
 */
#ifndef OCTAX_ORACLE_H
#define OCTAX_ORACLE_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- reward / termination descriptor (§3.3, App. C) ---------------------- */
enum { ORC_SRC_REG = 0, ORC_SRC_MEM = 1 };
enum {
  ORC_X_RAW = 0,            /* v                               */
  ORC_X_NEG = 1,            /* -v                              */
  ORC_X_DEC_TENS = 2,       /* v / 10                          */
  ORC_X_DEC_ONES = 3,       /* v % 10                          */
  ORC_X_DEC_TENS_MINUS_ONES = 4, /* v/10 - v%10   (Pong, §3.3)  */
  ORC_X_NIB_HI_MINUS_LO = 5,     /* (v>>4) - (v&15)             */
  ORC_X_ZERO_IF_GT = 6      /* v > arg ? 0 : v (Shooting Stars) */
};
enum { ORC_EQ = 0, ORC_NE = 1, ORC_GE = 2, ORC_GT = 3, ORC_LE = 4, ORC_LT = 5 };

typedef struct {
  int32_t src;    /* ORC_SRC_REG: V[idx]; ORC_SRC_MEM: RAM[idx & 0xFFF] */
  int32_t idx;
  int32_t xform;
  int32_t arg;
} orc_term;

typedef struct {
  orc_term lhs;
  int32_t cmp;
  int32_t rhs;
} orc_clause;

typedef struct {
  const uint8_t *rom;       /* program bytes, loaded at 0x200 */
  uint32_t rom_len;         /* 1 .. 3584 */
  uint32_t instr_per_frame; /* K */
  uint32_t frameskip;       /* frames per environment step */
  uint32_t stack_frames;    /* observation frames (<= frameskip) */
  uint32_t n_actions;       /* action index n_actions is the no-op */
  uint8_t action_set[16];   /* action index -> CHIP-8 key */
  uint32_t n_score_terms;   /* score = sum of terms (0 terms: score 0) */
  orc_term score[4];
  uint32_t n_term_clauses;  /* terminated = OR of clauses (0: never) */
  orc_clause term[4];
  uint32_t max_episode_steps; /* truncation; 0 = none */
  uint32_t startup_instrs;    /* instructions run at reset, no key held */
  uint32_t sticky_threshold;  /* sticky actions: repeat the previous action when
                                 a uniform 32-bit draw is below this; 0 = off */
  uint32_t max_noops;         /* no-op reset: 0..max_noops no-key steps after
                                 the startup instructions; 0 = off */
  uint32_t variant;           /* ORC_CHIP8 or ORC_SCHIP; one per environment */
} orc_game;

enum { ORC_CHIP8 = 0, ORC_SCHIP = 1 };

/* ---- status bits (sticky since creation) --------------------------------- */
enum { ORC_ST_BAD_OP = 1, ORC_ST_STACK_FAULT = 2, ORC_ST_BAD_ACTION = 4, ORC_ST_EXIT = 8 };

/* ---- one emulator instance ----------------------------------------------- */
typedef struct {
  uint8_t V[16];
  uint16_t I;
  uint16_t PC;
  uint8_t SP;          /* occupied stack entries, 0..16 */
  uint8_t DT, ST;
  uint8_t status;
  uint16_t stack[16];
  uint8_t pix[64][128]; /* one byte per pixel, 0 or 1, [y][x]; CHIP-8 uses
                           rows 0-31, columns 0-63 */
  uint8_t ram[4096];
  uint32_t episode_steps;
  uint32_t env_steps;
  /* random-number identity (CXNN) */
  uint32_t key[2];     /* Philox key = (seed low word, seed high word) */
  uint32_t uid;        /* instance identity, counter word 0 */
  uint32_t phase;      /* counter word 3: 0 = env step, 1 = reset startup */
  uint32_t draws;      /* CXNN draws so far in this step / startup */
  int32_t game;        /* index of this instance's game */
  uint8_t last_action; /* action index applied at the previous step (sticky) */
  uint8_t variant;     /* ORC_CHIP8 / ORC_SCHIP (copied from the game at reset) */
  uint8_t hires;       /* SCHIP: 1 = 128x64 mode, 0 = 64x32 mode (2x2 pixels) */
  uint8_t rpl[16];     /* SCHIP FX75/FX85 flag registers */
} orc_inst;

/* Canonical state record: the unit of comparison between implementations. */
typedef struct {
  uint8_t V[16];
  uint16_t I, PC;
  uint8_t SP, DT, ST, status;
  uint16_t stack[16];
  uint64_t display[64][2]; /* bit (x mod 64) of display[y][x / 64] = pixel (x, y);
                              CHIP-8 fills rows 0-31, word 0 */
  uint8_t ram[4096];
  uint32_t episode_steps, env_steps;
  uint8_t last_action;
  uint8_t hires;
  uint8_t pad[6];
  uint8_t rpl[16];
} orc_record;           /* 5208 bytes */

/* Bytes of one observation frame: 32*64 (CHIP-8) or 64*128 (SCHIP). */
size_t orc_frame_bytes(uint32_t variant);

/* Philox4x32-10 (Salmon et al., SC'11): out = bijection(counter; key). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* FNV-1a 64-bit over a byte string (Fowler/Noll/Vo). */
uint64_t orc_fnv1a64(const uint8_t *p, size_t n);

/* Single-instance primitives. */
int orc_inst_reset(orc_inst *m, const orc_game *g, uint32_t quirks);
void orc_exec_one(orc_inst *m, uint32_t quirks, int key_held /* -1 = none */);
void orc_tick_timers(orc_inst *m);
int32_t orc_score(const orc_inst *m, const orc_game *g);
int orc_terminated(const orc_inst *m, const orc_game *g);
int orc_inst_step(orc_inst *m, const orc_game *g, uint32_t quirks, uint32_t action,
                  uint8_t *obs /* stack_frames*32*64, nullable */, float *reward,
                  uint8_t *done);
void orc_inst_record(const orc_inst *m, orc_record *out);
uint64_t orc_inst_hash(const orc_inst *m);

/* A batch of independent instances (the loop over environments). */
typedef struct orc_env orc_env;
orc_env *orc_env_create(const orc_game *games, int n_games,
                        const uint16_t *game_of_env, /* nullable: all game 0 */
                        const uint32_t *uid_of_env,  /* nullable: uid = index */
                        int64_t n_envs, uint32_t quirks, uint64_t seed);
int orc_env_reset(orc_env *e, const uint8_t *mask /* nullable = all */,
                  uint8_t *obs /* [n][S][32][64], nullable */);
int orc_env_step(orc_env *e, const uint8_t *actions, uint8_t *obs, float *reward,
                 uint8_t *done, int n_threads);
int orc_env_hash(const orc_env *e, uint64_t *out);
int orc_env_records(const orc_env *e, orc_record *out);
orc_inst *orc_env_inst(orc_env *e, int64_t i);
int64_t orc_env_size(const orc_env *e);
void orc_env_destroy(orc_env *e);

/* Convenience: create a batch, run n_steps steps with actions[n_steps][n] and
 * collect per-step outputs (each nullable). Used for the CPU baseline. */
int orc_env_rollout(orc_env *e, int n_steps, const uint8_t *actions,
                    uint8_t *obs, float *reward, uint8_t *done,
                    uint64_t *hashes, int n_threads);

#ifdef __cplusplus
}
#endif
#endif
