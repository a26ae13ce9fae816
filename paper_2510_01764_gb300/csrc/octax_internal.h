// Internal declarations shared by the liboctax translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "octax.h"

namespace octax {

constexpr int kRamBytes = 4096;
constexpr int kPageShift = 6;               // 64-byte RAM pages: 64 pages -> one u64 mask
// Written-address range of an instance, lo | hi << 16 (lo > hi: nothing written).
constexpr uint32_t kNoWrites = 0x0FFFu;
constexpr int kFrameBytes = 32 * 64;        // one uint8 CHIP-8 observation frame
constexpr int kSchipFrameBytes = 64 * 128;  // one uint8 SCHIP observation frame (the 128x64 buffer)
constexpr uint32_t kBigFontAddr = 0x0A0;    // SCHIP 8x10 glyphs, 10 bytes each
// Packed display words (u64) per instance: 32 rows x 1 (CHIP-8), 64 rows x 2 (SCHIP).
constexpr int kDispWords = 32;
constexpr int kSchipDispWords = 128;
__host__ __device__ inline int frame_bytes(int schip) { return schip ? kSchipFrameBytes : kFrameBytes; }
__host__ __device__ inline int disp_words(int schip) { return schip ? kSchipDispWords : kDispWords; }
// A packed observation frame: the display words themselves (u64, bit x of a
// word = pixel x of its 64-pixel run).
__host__ __device__ inline int packed_frame_bytes(int schip) { return 8 * disp_words(schip); }
constexpr int kMaxBlock = 256;

// Game descriptor as the kernels read it (one per game, device memory).
struct TermDev {
  uint8_t src, xform;
  uint16_t idx;
  int32_t arg;
};
struct ClauseDev {
  TermDev lhs;
  int32_t cmp;
  int32_t rhs;
};
struct alignas(16) GameDev {
  uint32_t K, frameskip, n_actions, n_score, n_term, max_steps, startup, sticky;
  uint32_t max_noops, variant, pad[2];
  uint8_t action_set[16];
  TermDev score[4];
  ClauseDev term[4];
};
static_assert(sizeof(GameDev) <= 192, "GameDev must fit its shared-memory slot");
constexpr int kGameSmem = 192;
// Micro-op table: one entry per even address, 16 bytes (wide: operand offsets
// and NNN ready to use) or 8 bytes (narrow: packed; half the shared memory).
constexpr int kUopSmemWide = kRamBytes / 2 * 16;
constexpr int kUopSmemNarrow = kRamBytes / 2 * 8;
constexpr int kLutSmem = 256 * 8;            // byte of pixels -> 8 output bytes
constexpr int kAluSmem = 16 * 2 * 16;        // 8XYN coefficients per N (two int4)

// Emulator state, structure-of-arrays over slots (slot = index in these arrays).
struct DevState {
  int64_t n;              // slots
  uint32_t *v;            // [4][n]   V[4j..4j+3] little-endian in word j
  uint32_t *pcI;          // [n]      PC | I << 16
  uint32_t *misc;         // [n]      SP | DT << 8 | ST << 16 | status << 24
  uint16_t *stack;        // [16][n]
  uint64_t *disp;         // [W][n]   CHIP-8 (W = 32): bit x of word y = pixel (x, y);
                          //          SCHIP (W = 128): bit x of word 2y + h = pixel (64h + x, y)
  uint64_t *dirty;        // [n]      RAM pages that differ from the ROM image
  uint32_t *wrange;       // [n]      lowest | highest << 16 RAM address written since the
                          //          reset (kNoWrites: none): bytes outside it equal the image
  uint8_t *ram;           // [n][4096] per-instance RAM (valid on dirty pages only)
  uint32_t *ep;           // [n]      steps since reset
  uint32_t *env_steps;    // [n]      steps since creation
  int32_t *prev_score;    // [n]      score at the end of the last step / reset
  uint32_t *key;          // [2][n]   Philox key
  uint32_t *uid;          // [n]      Philox counter word 0
  uint32_t *out_row;      // [n]      row of this slot in its request's outputs
  uint16_t *game;         // [n]
  uint8_t *last_act;      // [n]      action index applied at the previous step
  uint8_t *mode;          // [n]      SCHIP: 1 = hires
  uint8_t *rpl;           // [n][16]  SCHIP flag registers
  int schip;              // 1: SCHIP layout (disp has 128 words per slot)
};

// Every per-slot array is set (checked on the host before each launch).
inline bool state_complete(const DevState &s) {
  return s.n > 0 && s.v && s.pcI && s.misc && s.stack && s.disp && s.dirty && s.wrange && s.ram && s.ep && s.env_steps &&
         s.prev_score && s.key && s.uid && s.out_row && s.game && s.last_act && s.mode && s.rpl;
}

// A group: up to block/32*ipw consecutive slots that share one game (one CTA's work).
struct Group {
  uint32_t slot0;
  uint16_t count;
  uint16_t game;
  uint32_t io;            // index into the IO table (0 when launched with io0)
  uint32_t row0;          // output row of slot0 within its request (serving resets)
};

// Where one request's per-step inputs and outputs live.
struct IO {
  const uint8_t *actions;  // [steps][rows]
  uint8_t *obs;            // [steps][rows][S][H][W]
  float *reward;           // [steps][rows]
  uint8_t *done;           // [steps][rows]
  int64_t rows;            // rows per step
  int32_t packed;          // 1: obs frames are the packed display words (packed_frame_bytes)
  int32_t pad;
};

struct StepLaunch {
  DevState st;
  const GameDev *games;
  const uint8_t *images;   // [n_games][4096] initial RAM image (font + ROM)
  const Group *groups;
  int n_groups;
  IO io0;                  // used when io_table == nullptr
  const IO *io_table;
  int step0;               // output step index of this launch's first step
  int steps;               // env steps in this launch
  int S;                   // stack frames
  uint32_t quirks;
  int ipw;                 // instances emulated per warp (1..32)
  int writers;             // >0: warp-specialised kernel with this many writer warps
  unsigned int *work_counter;  // non-null: persistent CTAs pull groups from it
  unsigned int *err;       // set when a bounded barrier wait gives up (specialised kernel)
  int wrappers;            // 1: some game uses sticky actions or no-op reset (kernel variant)
  int stall_writers;       // diagnostic: writer warps skip the hand-over (specialised kernel)
};

struct ResetLaunch {
  DevState st;
  const GameDev *games;
  const uint8_t *images;
  const Group *groups;
  int n_groups;
  const uint8_t *mask;     // [n_out_rows] by out_row, nullable = all
  uint8_t *obs;            // [rows][S][32][64] by out_row, nullable
  int S;
  uint32_t quirks;
  int ipw;
  int init;                // 1: also set key/uid/env_steps/status (creation)
  uint64_t seed;
  const uint32_t *uid_of_slot;  // used when init (nullable = out_row)
  const uint64_t *seed_of_group;  // init: per-group seed (nullable = seed)
  int set_rows;            // init: out_row = group.row0 + lane, game = group.game
};

// Dynamic shared memory of a step CTA; wide = 16-byte micro-op table (the
// narrow size is the minimum a launch shape needs).
size_t step_smem_bytes(int block, int ipw, int schip, int wide = 0);
// Warp-specialised kernel: `block` emulator threads plus 32 * writers writer threads.
size_t step_ws_smem_bytes(int block, int ipw);
size_t max_dynamic_smem();
cudaError_t launch_step(const StepLaunch &p, int grid, int block, cudaStream_t s);
cudaError_t launch_reset(const ResetLaunch &p, int block, cudaStream_t s);
cudaError_t launch_hash(const DevState &st, const uint8_t *images, const uint32_t *slot_of_row,
                        int64_t rows, uint64_t *out, cudaStream_t s);
cudaError_t launch_records(const DevState &st, const uint8_t *images, const uint32_t *slot_of_row,
                           int64_t first, int64_t count, octax_state_record *out, cudaStream_t s);
cudaError_t launch_set_records(const DevState &st, const GameDev *games, const uint8_t *images,
                               const uint32_t *slot_of_row, int64_t first, int64_t count,
                               const octax_state_record *in, cudaStream_t s);
int max_resident_ctas(int block, int ipw, int writers, int wrappers, int schip);
// True when a game enables the sticky-action or no-op-reset wrapper.
inline int uses_wrappers(const GameDev *games, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (games[i].sticky != 0u || games[i].max_noops != 0u) return 1;
  return 0;
}
// Bytes of device state per slot (all DevState arrays).
constexpr size_t kSlotStateBytes = 16 + 4 + 4 + 32 + 256 + 8 + 4 + 4096 + 4 + 4 + 4 + 8 + 4 + 4 + 2 + 1 + 1 + 16;
inline size_t slot_state_bytes(int schip) {
  return kSlotStateBytes + (schip ? 8 * (kSchipDispWords - kDispWords) : 0);
}
cudaError_t alloc_state(DevState &st, int64_t n, int schip, void **block_out, size_t *bytes_out);
// Append one step launch to a graph (after `dep`, if non-null).
cudaError_t add_step_node(cudaGraph_t g, cudaGraphNode_t *node, cudaGraphNode_t dep, const StepLaunch &p,
                          int grid, int block);

// Validate game descriptors; build device descriptors and 4 KB RAM images.
int build_games(const octax_game *games, int n_games, std::vector<GameDev> &dev,
                std::vector<uint8_t> &images);

// Error reporting (thread-local message).
void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

}  // namespace octax
