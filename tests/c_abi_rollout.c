/*
 * A C program that uses liboctax through include/octax.h alone: no CUDA
 * runtime calls and no Python. It loads a ROM file, creates n environments of
 * one game, steps them with host buffers (octax_step_host) and prints, per
 * instance, the FNV-1a 64 hash of its canonical state record, then the sums of
 * rewards and done flags. tests/test_c_abi.py compiles it, runs it and checks
 * the hashes against the CPU oracle.
 *
 * usage: c_abi_rollout ROM N_ENVS N_STEPS SEED [packed]
 * actions: instance i at step s takes index (7 i + 3 s) mod 5 (4 is the no-op).
 * With "packed" it steps through octax_step_host_packed (one bit per pixel)
 * and also prints the sum of the set observation bits of the last step.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "octax.h"

static uint64_t fnv_bytes(uint64_t h, const void *p, size_t n) {
  const uint8_t *b = (const uint8_t *)p;
  for (size_t i = 0; i < n; i++) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

/* The hashed serialisation of a CHIP-8 record: V, I, PC, SP, DT, ST, status,
 * stack, display rows 0-31 (word 0), ram, episode_steps, env_steps,
 * last_action (little-endian host assumed, as on x86-64 and aarch64). */
static uint64_t record_hash(const octax_state_record *r) {
  uint64_t h = 14695981039346656037ull;
  h = fnv_bytes(h, r->V, 16);
  h = fnv_bytes(h, &r->I, 2);
  h = fnv_bytes(h, &r->PC, 2);
  h = fnv_bytes(h, &r->SP, 1);
  h = fnv_bytes(h, &r->DT, 1);
  h = fnv_bytes(h, &r->ST, 1);
  h = fnv_bytes(h, &r->status, 1);
  h = fnv_bytes(h, r->stack, 32);
  for (int y = 0; y < 32; y++) h = fnv_bytes(h, &r->display[y][0], 8);
  h = fnv_bytes(h, r->ram, 4096);
  h = fnv_bytes(h, &r->episode_steps, 4);
  h = fnv_bytes(h, &r->env_steps, 4);
  h = fnv_bytes(h, &r->last_action, 1);
  return h;
}

int main(int argc, char **argv) {
  if (argc != 5 && !(argc == 6 && strcmp(argv[5], "packed") == 0)) {
    fprintf(stderr, "usage: %s ROM N_ENVS N_STEPS SEED [packed]\n", argv[0]);
    return 2;
  }
  const int packed = argc == 6;
  FILE *f = fopen(argv[1], "rb");
  if (!f) {
    perror("rom");
    return 2;
  }
  static uint8_t rom[3584];
  const size_t rom_len = fread(rom, 1, sizeof rom, f);
  fclose(f);
  const int64_t n = atoll(argv[2]);
  const int steps = atoi(argv[3]);
  const uint64_t seed = strtoull(argv[4], NULL, 10);

  octax_game g;
  memset(&g, 0, sizeof g);
  g.rom = rom;
  g.rom_len = (uint32_t)rom_len;
  g.instr_per_frame = 10;
  g.frameskip = 4;
  g.stack_frames = 4;
  g.n_actions = 4;
  const uint8_t keys[4] = {7, 9, 5, 8};
  memcpy(g.action_set, keys, 4);
  g.n_score_terms = 1;
  g.score[0].src = OCTAX_SRC_REG;
  g.score[0].idx = 6;
  g.score[0].xform = OCTAX_X_RAW;
  g.n_term_clauses = 1;
  g.term[0].lhs.src = OCTAX_SRC_REG;
  g.term[0].lhs.idx = 6;
  g.term[0].lhs.xform = OCTAX_X_RAW;
  g.term[0].cmp = OCTAX_CMP_GE;
  g.term[0].rhs = 3;
  g.variant = OCTAX_VARIANT_CHIP8;

  octax_env *env = NULL;
  if (octax_create(&g, 1, NULL, NULL, n, 0, seed, NULL, &env) != OCTAX_OK) {
    fprintf(stderr, "octax_create: %s\n", octax_last_error());
    return 1;
  }
  uint8_t *actions = malloc((size_t)n);
  uint8_t *obs = malloc((size_t)n * 4 * 32 * 64);
  uint64_t *obs_words = malloc((size_t)n * 4 * 32 * sizeof(uint64_t));
  float *reward = malloc((size_t)n * sizeof(float));
  uint8_t *done = malloc((size_t)n);
  octax_state_record *recs = malloc((size_t)n * sizeof(octax_state_record));
  double reward_sum = 0;
  long done_sum = 0;
  for (int s = 0; s < steps; s++) {
    for (int64_t i = 0; i < n; i++) actions[i] = (uint8_t)((7 * i + 3 * s) % 5);
    const int rc = packed ? octax_step_host_packed(env, actions, obs_words, reward, done)
                          : octax_step_host(env, actions, obs, reward, done);
    if (rc != OCTAX_OK) {
      fprintf(stderr, "step: %s\n", octax_last_error());
      return 1;
    }
    for (int64_t i = 0; i < n; i++) {
      reward_sum += reward[i];
      done_sum += done[i];
    }
  }
  if (octax_get_state(env, 0, n, recs) != OCTAX_OK) {
    fprintf(stderr, "octax_get_state: %s\n", octax_last_error());
    return 1;
  }
  for (int64_t i = 0; i < n; i++) printf("%016llx\n", (unsigned long long)record_hash(&recs[i]));
  long lit = 0;
  if (packed) {
    for (size_t k = 0; k < (size_t)n * 4 * 32; k++)
      for (uint64_t w = obs_words[k]; w; w &= w - 1) lit++;
  } else {
    for (size_t k = 0; k < (size_t)n * 4 * 32 * 64; k++) lit += obs[k];
  }
  printf("reward %.0f done %ld lit %ld\n", reward_sum, done_sum, lit);
  octax_destroy(env);
  free(actions);
  free(obs);
  free(obs_words);
  free(reward);
  free(done);
  free(recs);
  return 0;
}
