// liboctax host side: the C-ABI declared in include/octax.h.
//
// An environment owns its emulator state (structure-of-arrays over "slots";
// slots are instances sorted by game so that every CTA runs one game), the
// per-game descriptors and 4 KB initial RAM images, the group tables for each
// CTA size, and a cache of explicitly built CUDA graphs for octax_step_n.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "octax_internal.h"

namespace octax {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char *what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return OCTAX_ECUDA;
}

// The conventional 4x5 hexadecimal font, 5 bytes per glyph, loaded at 0x050
// (the paper fixes the location 0x050-0x09F; the glyph shapes are the
// customary CHIP-8 ones).
static const uint8_t kFont[80] = {
    0xF0, 0x90, 0x90, 0x90, 0xF0, 0x20, 0x60, 0x20, 0x20, 0x70, 0xF0, 0x10, 0xF0, 0x80,
    0xF0, 0xF0, 0x10, 0xF0, 0x10, 0xF0, 0x90, 0x90, 0xF0, 0x10, 0x10, 0xF0, 0x80, 0xF0,
    0x10, 0xF0, 0xF0, 0x80, 0xF0, 0x90, 0xF0, 0xF0, 0x10, 0x20, 0x40, 0x40, 0xF0, 0x90,
    0xF0, 0x90, 0xF0, 0xF0, 0x90, 0xF0, 0x10, 0xF0, 0xF0, 0x90, 0xF0, 0x90, 0x90, 0xE0,
    0x90, 0xE0, 0x90, 0xE0, 0xF0, 0x80, 0x80, 0x80, 0xF0, 0xE0, 0x90, 0x90, 0x90, 0xE0,
    0xF0, 0x80, 0xF0, 0x80, 0xF0, 0xF0, 0x80, 0xF0, 0x80, 0x80};

}  // namespace octax

using namespace octax;

struct GroupTable {
  Group *dev = nullptr;
  int count = 0;
};

struct GraphKey {
  int n_steps, block, ipw, spl, persistent, writers, balance;
  bool operator<(const GraphKey &o) const {
    return std::tie(n_steps, block, ipw, spl, persistent, writers, balance) <
           std::tie(o.n_steps, o.block, o.ipw, o.spl, o.persistent, o.writers, o.balance);
  }
};

struct octax_env {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t n = 0;
  int n_games = 0;
  int S = 4;
  int schip = 0;  // OCTAX_VARIANT_SCHIP environment
  uint32_t quirks = 0;
  uint64_t seed = 0;
  std::vector<GameDev> games_h;
  std::vector<uint16_t> game_of_slot;
  GameDev *games_d = nullptr;
  uint8_t *images_d = nullptr;
  DevState st{};
  uint32_t *slot_of_row_d = nullptr;
  std::vector<void *> allocs;
  size_t bytes = 0;
  octax_launch cfg{64, 8, 4, 0, 1, 0, 0};
  std::map<std::pair<int, int>, GroupTable> groups;  // by (instances per CTA, wave)
  unsigned int *counters_d = nullptr;
  int counters_cap = 0;
  IO *io_d = nullptr;
  unsigned int *err_d = nullptr;  // set by a kernel whose bounded hand-over wait gave up
  int stall_writers = 0;          // octax_debug_stall_writers
  std::map<GraphKey, cudaGraphExec_t> graphs;
  // octax_step_host staging
  uint8_t *hs_act = nullptr, *hs_obs = nullptr, *hs_done = nullptr;
  float *hs_rew = nullptr;
  cudaEvent_t ev = nullptr;
};

namespace {

template <class T>
cudaError_t dalloc(octax_env *e, T **p, size_t count) {
  void *q = nullptr;
  const size_t bytes = count * sizeof(T);
  cudaError_t r = cudaMalloc(&q, bytes > 0 ? bytes : 16);
  if (r != cudaSuccess) return r;
  e->allocs.push_back(q);
  e->bytes += bytes;
  *p = static_cast<T *>(q);
  return cudaSuccess;
}

int validate_game(const octax_game &g, int S, int variant) {
  char buf[160];
  if (!g.rom || g.rom_len < 1 || g.rom_len > 3584) {
    set_error("game rom must be 1..3584 bytes");
    return OCTAX_EINVAL;
  }
  if (g.instr_per_frame < 1 || g.frameskip < 1 || g.stack_frames < 1 || g.stack_frames > g.frameskip) {
    set_error("need instr_per_frame >= 1, frameskip >= 1, 1 <= stack_frames <= frameskip");
    return OCTAX_EINVAL;
  }
  if (g.stack_frames != S) {
    set_error("all games of one environment need the same stack_frames");
    return OCTAX_EINVAL;
  }
  if (g.variant > OCTAX_VARIANT_SCHIP || g.variant != variant) {
    set_error("variant must be OCTAX_VARIANT_CHIP8 or OCTAX_VARIANT_SCHIP, the same for all games");
    return OCTAX_EINVAL;
  }
  if (g.max_noops > 255u) {
    set_error("max_noops must be <= 255");
    return OCTAX_EINVAL;
  }
  if (g.startup_instrs > (1u << 20)) {
    set_error("startup_instrs must be <= 2^20");
    return OCTAX_EINVAL;
  }
  if (g.n_actions > 16 || g.n_score_terms > 4 || g.n_term_clauses > 4) {
    set_error("n_actions <= 16, n_score_terms <= 4, n_term_clauses <= 4");
    return OCTAX_EINVAL;
  }
  for (int i = 0; i < g.n_actions; ++i)
    if (g.action_set[i] > 15) {
      snprintf(buf, sizeof buf, "action_set[%d] = %d is not a CHIP-8 key", i, g.action_set[i]);
      set_error(buf);
      return OCTAX_EINVAL;
    }
  auto bad_term = [](const octax_term &t) { return t.src > OCTAX_SRC_MEM || t.xform > OCTAX_X_ZERO_IF_GT; };
  for (int i = 0; i < g.n_score_terms; ++i)
    if (bad_term(g.score[i])) {
      set_error("score term: bad src or xform");
      return OCTAX_EINVAL;
    }
  for (int i = 0; i < g.n_term_clauses; ++i)
    if (bad_term(g.term[i].lhs) || g.term[i].cmp > OCTAX_CMP_LT) {
      set_error("termination clause: bad src, xform or cmp");
      return OCTAX_EINVAL;
    }
  return OCTAX_OK;
}

GameDev to_dev(const octax_game &g) {
  GameDev d;
  memset(&d, 0, sizeof d);
  d.K = g.instr_per_frame;
  d.frameskip = g.frameskip;
  d.n_actions = g.n_actions;
  d.n_score = g.n_score_terms;
  d.n_term = g.n_term_clauses;
  d.max_steps = g.max_episode_steps;
  d.startup = g.startup_instrs;
  d.sticky = g.sticky_threshold;
  d.max_noops = g.max_noops;
  d.variant = g.variant;
  memcpy(d.action_set, g.action_set, 16);
  for (int i = 0; i < 4; ++i) {
    d.score[i] = TermDev{g.score[i].src, g.score[i].xform, g.score[i].idx, g.score[i].arg};
    d.term[i].lhs = TermDev{g.term[i].lhs.src, g.term[i].lhs.xform, g.term[i].lhs.idx, g.term[i].lhs.arg};
    d.term[i].cmp = g.term[i].cmp;
    d.term[i].rhs = g.term[i].rhs;
  }
  return d;
}

int block_ok(int b) { return b == 32 || b == 64 || b == 128 || b == 256; }
int ipw_ok(int v) { return v >= 1 && v <= 32; }
int per_cta(const octax_launch &c) { return c.block / 32 * c.inst_per_warp; }

// Resident CTAs of one wave for a balanced launch (0 = not balanced).
int wave_of(const octax_env *e, const octax_launch &c) {
  if (!c.balance) return 0;
  return max_resident_ctas(c.block, c.inst_per_warp, c.writer_warps,
                           uses_wrappers(e->games_h.data(), e->games_h.size()), e->schip);
}

const char *launch_problem(const octax_launch &c, int schip) {
  if (!block_ok(c.block) || !ipw_ok(c.inst_per_warp)) return "block in {32,64,128,256}, inst_per_warp in {1,...,32}";
  if (c.steps_per_launch < 1 || c.steps_per_launch > 256) return "steps_per_launch 1..256";
  if ((c.persistent != 0 && c.persistent != 1) || (c.use_graph != 0 && c.use_graph != 1) ||
      (c.balance != 0 && c.balance != 1))
    return "flags 0/1";
  if (c.writer_warps != 0) {
    const int W = c.writer_warps, J = per_cta(c);
    if (!(W == 1 || W == 2 || W == 4 || W == 8)) return "writer_warps in {0,1,2,4,8}";
    if (J % W != 0 || !(J / W == 8 || J / W == 16 || J / W == 32))
      return "block/32*inst_per_warp/writer_warps must be 8, 16 or 32";
    if (schip) return "writer warps serve CHIP-8 environments only";
    if (step_ws_smem_bytes(c.block, c.inst_per_warp) > max_dynamic_smem())
      return "too many instances per CTA for the writer ring";
  }
  if (step_smem_bytes(c.block, c.inst_per_warp, schip) > max_dynamic_smem())
    return "too many instances per CTA for shared memory";
  return nullptr;
}

}  // namespace

// Validate the descriptors and build the device descriptors + initial RAM images.
int octax::build_games(const octax_game *games, int n_games, std::vector<GameDev> &dev,
                       std::vector<uint8_t> &images) {
  for (int g = 0; g < n_games; ++g) {
    int rc = validate_game(games[g], games[0].stack_frames, games[0].variant);
    if (rc) return rc;
  }
  dev.clear();
  images.assign((size_t)n_games * kRamBytes, 0);
  for (int g = 0; g < n_games; ++g) {
    dev.push_back(to_dev(games[g]));
    uint8_t *img = &images[(size_t)g * kRamBytes];
    memcpy(img + 0x50, kFont, sizeof kFont);
    if (games[g].variant == OCTAX_VARIANT_SCHIP)
      // 8x10 glyphs: glyph pixel (c, r) of the 4x5 font drawn as the 2x2 block
      // at columns 2c, 2c+1 of rows 2r, 2r+1 (MSB = leftmost pixel).
      for (int d = 0; d < 16; ++d)
        for (int r = 0; r < 10; ++r) {
          uint8_t out = 0;
          for (int c = 0; c < 4; ++c)
            if (kFont[5 * d + r / 2] & (0x80 >> c)) out |= (uint8_t)(0xC0 >> (2 * c));
          img[kBigFontAddr + 10 * d + r] = out;
        }
    memcpy(img + 0x200, games[g].rom, games[g].rom_len);
  }
  return OCTAX_OK;
}

namespace {

// Groups of up to `cap` (instances per CTA) consecutive same-game slots.
// wave > 0 (balanced): the group count is rounded up to a whole number of
// waves of `wave` resident CTAs and every run of same-game slots is cut into
// groups of near-equal size, so that every SM receives the same number of
// CTAs of about the same size. wave = 0: full groups, a ragged last one.
int get_groups(octax_env *e, int cap, int wave, GroupTable **out) {
  const std::pair<int, int> gkey(cap, wave);
  auto it = e->groups.find(gkey);
  if (it != e->groups.end()) {
    *out = &it->second;
    return OCTAX_OK;
  }
  std::vector<std::pair<int64_t, int64_t>> runs;  // [first, end) of same-game slots
  for (int64_t s = 0; s < e->n;) {
    int64_t end = s;
    while (end < e->n && e->game_of_slot[end] == e->game_of_slot[s]) ++end;
    runs.emplace_back(s, end);
    s = end;
  }
  int64_t size = cap;  // target instances per group
  if (wave > 0) {
    int64_t g0 = 0;
    for (const auto &r : runs) g0 += (r.second - r.first + cap - 1) / cap;
    const int64_t g = (g0 + wave - 1) / wave * wave;
    size = std::max<int64_t>(1, (e->n + g - 1) / g);  // <= cap because g >= g0
  }
  std::vector<Group> gs;
  for (const auto &r : runs) {
    const int64_t len = r.second - r.first, k = (len + size - 1) / size;
    const uint16_t game = e->game_of_slot[r.first];
    int64_t s = r.first;
    for (int64_t q = 0; q < k; ++q) {
      const int64_t cnt = len / k + (q < len % k ? 1 : 0);
      gs.push_back(Group{(uint32_t)s, (uint16_t)cnt, game, 0u, 0u});
      s += cnt;
    }
  }
  // Longest first (instructions per step): CTAs are dispatched, and the
  // persistent queue hands out groups, in table order.
  std::stable_sort(gs.begin(), gs.end(), [&](const Group &a, const Group &b) {
    const uint32_t ca = e->games_h[a.game].K * e->games_h[a.game].frameskip;
    const uint32_t cb = e->games_h[b.game].K * e->games_h[b.game].frameskip;
    return ca > cb;
  });
  GroupTable t;
  t.count = (int)gs.size();
  cudaError_t r = dalloc(e, &t.dev, gs.size());
  if (r != cudaSuccess) return cuda_fail(r, "group table");
  r = cudaMemcpy(t.dev, gs.data(), gs.size() * sizeof(Group), cudaMemcpyHostToDevice);
  if (r != cudaSuccess) return cuda_fail(r, "group table upload");
  e->groups[gkey] = t;
  *out = &e->groups[gkey];
  return OCTAX_OK;
}

int ensure_counters(octax_env *e, int count) {
  if (count <= e->counters_cap) return OCTAX_OK;
  unsigned int *p = nullptr;
  cudaError_t r = dalloc(e, &p, (size_t)count);
  if (r != cudaSuccess) return cuda_fail(r, "work counters");
  e->counters_d = p;
  e->counters_cap = count;
  return OCTAX_OK;
}

StepLaunch base_launch(octax_env *e, const GroupTable *gt) {
  StepLaunch p;
  memset(&p, 0, sizeof p);
  p.st = e->st;
  p.games = e->games_d;
  p.images = e->images_d;
  p.groups = gt->dev;
  p.n_groups = gt->count;
  p.S = e->S;
  p.quirks = e->quirks;
  p.ipw = e->cfg.inst_per_warp;
  p.err = e->err_d;
  p.wrappers = uses_wrappers(e->games_h.data(), e->games_h.size());
  p.stall_writers = e->stall_writers;
  return p;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int check_io(const uint8_t *actions, const uint8_t *obs, const float *reward, const uint8_t *done) {
  if (!actions || !obs || !reward || !done) {
    set_error("actions, obs, reward and done must be non-null device pointers");
    return OCTAX_EINVAL;
  }
  if (!aligned16(obs)) {
    set_error("obs must be 16-byte aligned");
    return OCTAX_EINVAL;
  }
  return OCTAX_OK;
}

// Enqueue n_steps steps as a chain of launches of `spl` steps each.
int enqueue_steps(octax_env *e, const octax_launch &cfg, int n_steps, const IO &io) {
  GroupTable *gt = nullptr;
  int rc = get_groups(e, per_cta(cfg), wave_of(e, cfg), &gt);
  if (rc) return rc;
  const int spl = cfg.steps_per_launch;
  const int launches = (n_steps + spl - 1) / spl;
  const int grid =
      cfg.persistent
          ? std::min(gt->count, std::max(1, max_resident_ctas(cfg.block, cfg.inst_per_warp, cfg.writer_warps,
                                                      uses_wrappers(e->games_h.data(), e->games_h.size()),
                                                      e->schip)))
          : gt->count;
  if (cfg.persistent) {
    rc = ensure_counters(e, launches);
    if (rc) return rc;
  }
  if (!cfg.use_graph || launches == 1) {
    if (cfg.persistent) {
      cudaError_t r = cudaMemsetAsync(e->counters_d, 0, sizeof(unsigned) * launches, e->stream);
      if (r != cudaSuccess) return cuda_fail(r, "counter reset");
    }
    for (int j = 0; j < launches; ++j) {
      StepLaunch p = base_launch(e, gt);
      p.ipw = cfg.inst_per_warp;
      p.writers = cfg.writer_warps;
      p.io0 = io;
      p.step0 = j * spl;
      p.steps = std::min(spl, n_steps - j * spl);
      p.work_counter = cfg.persistent ? e->counters_d + j : nullptr;
      cudaError_t r = launch_step(p, grid, cfg.block, e->stream);
      if (r != cudaSuccess) return cuda_fail(r, "step launch");
    }
    return OCTAX_OK;
  }
  // CUDA graph: the kernels read their IO from io_d, refreshed before replay.
  const GraphKey key{n_steps, cfg.block, cfg.inst_per_warp, spl, cfg.persistent, cfg.writer_warps, cfg.balance};
  auto it = e->graphs.find(key);
  if (it == e->graphs.end()) {
    cudaGraph_t g;
    cudaError_t r = cudaGraphCreate(&g, 0);
    if (r != cudaSuccess) return cuda_fail(r, "graph create");
    cudaGraphNode_t prev = nullptr;
    if (cfg.persistent) {
      cudaMemsetParams mp;
      memset(&mp, 0, sizeof mp);
      mp.dst = e->counters_d;
      mp.value = 0;
      mp.elementSize = 4;
      mp.width = (size_t)launches;
      mp.height = 1;
      mp.pitch = 0;
      r = cudaGraphAddMemsetNode(&prev, g, nullptr, 0, &mp);
      if (r != cudaSuccess) return cuda_fail(r, "graph memset node");
    }
    for (int j = 0; j < launches; ++j) {
      StepLaunch p = base_launch(e, gt);
      p.ipw = cfg.inst_per_warp;
      p.writers = cfg.writer_warps;
      p.io_table = e->io_d;
      p.step0 = j * spl;
      p.steps = std::min(spl, n_steps - j * spl);
      p.work_counter = cfg.persistent ? e->counters_d + j : nullptr;
      cudaGraphNode_t node;
      r = add_step_node(g, &node, prev, p, grid, cfg.block);
      if (r != cudaSuccess) return cuda_fail(r, "graph kernel node");
      prev = node;
    }
    cudaGraphExec_t ex;
    r = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (r != cudaSuccess) return cuda_fail(r, "graph instantiate");
    it = e->graphs.emplace(key, ex).first;
  }
  // Pageable source: the runtime stages it before returning, so the stack copy is safe.
  IO io_copy = io;
  cudaError_t r = cudaMemcpyAsync(e->io_d, &io_copy, sizeof(IO), cudaMemcpyHostToDevice, e->stream);
  if (r != cudaSuccess) return cuda_fail(r, "io upload");
  r = cudaGraphLaunch(it->second, e->stream);
  if (r != cudaSuccess) return cuda_fail(r, "graph launch");
  return OCTAX_OK;
}

}  // namespace

namespace octax {
cudaStream_t env_stream(const octax_env *e) { return e ? e->stream : nullptr; }
int env_device(const octax_env *e) { return e ? e->device : -1; }
}  // namespace octax

namespace {

void free_env(octax_env *e) {
  if (!e) return;
  cudaSetDevice(e->device);
  if (e->stream) cudaStreamSynchronize(e->stream);
  for (auto &kv : e->graphs) cudaGraphExecDestroy(kv.second);
  for (void *p : e->allocs) cudaFree(p);
  if (e->ev) cudaEventDestroy(e->ev);
  if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
  delete e;
}

}  // namespace

extern "C" {

const char *octax_last_error(void) { return g_last_error.c_str(); }

int octax_create(const octax_game *games, int n_games, const uint16_t *game_of_env,
                 const uint32_t *uid_of_env, int64_t n_envs, uint32_t quirks, uint64_t seed,
                 void *cuda_stream, octax_env **out) {
  if (!out || !games || n_games < 1 || n_games > 65535 || n_envs < 1 || n_envs > (int64_t)1 << 31) {
    set_error("octax_create: need out, games, 1 <= n_games <= 65535, 1 <= n_envs <= 2^31");
    return OCTAX_EINVAL;
  }
  *out = nullptr;
  if (quirks & ~0x3Fu) {
    set_error("octax_create: unknown quirk bits");
    return OCTAX_EINVAL;
  }
  std::vector<GameDev> games_dev;
  std::vector<uint8_t> images;
  {
    int rc = build_games(games, n_games, games_dev, images);
    if (rc) return rc;
  }
  if (game_of_env)
    for (int64_t i = 0; i < n_envs; ++i)
      if (game_of_env[i] >= n_games) {
        set_error("octax_create: game_of_env entry out of range");
        return OCTAX_EINVAL;
      }
  octax_env *e = new octax_env();
  cudaGetDevice(&e->device);
  e->n = n_envs;
  e->n_games = n_games;
  e->S = games[0].stack_frames;
  e->schip = games[0].variant == OCTAX_VARIANT_SCHIP;
  e->quirks = quirks;
  e->seed = seed;
  if (cuda_stream) {
    e->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {  // blocking stream: ordered with the legacy default stream
    cudaError_t r = cudaStreamCreate(&e->stream);
    if (r != cudaSuccess) {
      free_env(e);
      return cuda_fail(r, "stream create");
    }
    e->own_stream = true;
  }
  // slots: instances stably sorted by game
  std::vector<uint32_t> slot_of_row(n_envs), row_of_slot(n_envs);
  std::iota(row_of_slot.begin(), row_of_slot.end(), 0u);
  if (game_of_env)
    std::stable_sort(row_of_slot.begin(), row_of_slot.end(),
                     [&](uint32_t a, uint32_t b) { return game_of_env[a] < game_of_env[b]; });
  e->game_of_slot.resize(n_envs);
  std::vector<uint32_t> uid_of_slot(n_envs);
  for (int64_t s = 0; s < n_envs; ++s) {
    const uint32_t row = row_of_slot[s];
    slot_of_row[row] = (uint32_t)s;
    e->game_of_slot[s] = game_of_env ? game_of_env[row] : 0;
    uid_of_slot[s] = uid_of_env ? uid_of_env[row] : row;
  }
  e->games_h = games_dev;
  const size_t n = (size_t)n_envs;
  DevState &st = e->st;
  st.n = n_envs;
  cudaError_t r = cudaSuccess;
  uint32_t *uid_tmp = nullptr;
#define ALLOC(ptr, cnt) \
  if (r == cudaSuccess) r = dalloc(e, &(ptr), (cnt))
  ALLOC(e->games_d, (size_t)n_games);
  ALLOC(e->images_d, images.size());
  ALLOC(st.v, 4 * n);
  ALLOC(st.pcI, n);
  ALLOC(st.misc, n);
  ALLOC(st.stack, 16 * n);
  ALLOC(st.disp, (size_t)disp_words(e->schip) * n);
  ALLOC(st.dirty, n);
  ALLOC(st.wrange, n);
  ALLOC(st.ram, n * kRamBytes);
  ALLOC(st.ep, n);
  ALLOC(st.env_steps, n);
  ALLOC(st.prev_score, n);
  ALLOC(st.key, 2 * n);
  ALLOC(st.uid, n);
  ALLOC(st.out_row, n);
  ALLOC(st.game, n);
  ALLOC(st.last_act, n);
  ALLOC(st.mode, n);
  ALLOC(st.rpl, 16 * n);
  st.schip = e->schip;
  ALLOC(e->slot_of_row_d, n);
  ALLOC(e->io_d, 1);
  ALLOC(e->err_d, 1);
  ALLOC(uid_tmp, n);
#undef ALLOC
  if (r != cudaSuccess) {
    free_env(e);
    set_error(std::string("octax_create: device allocation failed: ") + cudaGetErrorString(r));
    return OCTAX_ENOMEM;
  }
  r = cudaMemcpy(e->games_d, e->games_h.data(), e->games_h.size() * sizeof(GameDev), cudaMemcpyHostToDevice);
  if (r == cudaSuccess) r = cudaMemcpy(e->images_d, images.data(), images.size(), cudaMemcpyHostToDevice);
  if (r == cudaSuccess) r = cudaMemcpy(st.out_row, row_of_slot.data(), n * 4, cudaMemcpyHostToDevice);
  if (r == cudaSuccess) r = cudaMemcpy(st.game, e->game_of_slot.data(), n * 2, cudaMemcpyHostToDevice);
  if (r == cudaSuccess) r = cudaMemcpy(e->slot_of_row_d, slot_of_row.data(), n * 4, cudaMemcpyHostToDevice);
  if (r == cudaSuccess) r = cudaMemcpy(uid_tmp, uid_of_slot.data(), n * 4, cudaMemcpyHostToDevice);
  if (r == cudaSuccess) r = cudaMemset(e->err_d, 0, sizeof(unsigned int));
  if (r == cudaSuccess) r = cudaEventCreateWithFlags(&e->ev, cudaEventDisableTiming);
  if (r != cudaSuccess) {
    int rc = cuda_fail(r, "octax_create upload");
    free_env(e);
    return rc;
  }
  GroupTable *gt = nullptr;
  int rc = get_groups(e, per_cta(e->cfg), wave_of(e, e->cfg), &gt);
  if (rc) {
    free_env(e);
    return rc;
  }
  ResetLaunch p;
  memset(&p, 0, sizeof p);
  p.st = st;
  p.games = e->games_d;
  p.images = e->images_d;
  p.groups = gt->dev;
  p.n_groups = gt->count;
  p.S = e->S;
  p.quirks = quirks;
  p.ipw = e->cfg.inst_per_warp;
  p.init = 1;
  p.seed = seed;
  p.uid_of_slot = uid_tmp;
  r = launch_reset(p, e->cfg.block, e->stream);
  if (r == cudaSuccess) r = cudaStreamSynchronize(e->stream);
  if (r != cudaSuccess) {
    rc = cuda_fail(r, "octax_create reset");
    free_env(e);
    return rc;
  }
  *out = e;
  return OCTAX_OK;
}

int octax_reset(octax_env *e, const uint8_t *mask_dev, uint8_t *obs_dev) {
  if (!e) {
    set_error("octax_reset: null env");
    return OCTAX_EINVAL;
  }
  if (obs_dev && !aligned16(obs_dev)) {
    set_error("octax_reset: obs must be 16-byte aligned");
    return OCTAX_EINVAL;
  }
  GroupTable *gt = nullptr;
  int rc = get_groups(e, per_cta(e->cfg), wave_of(e, e->cfg), &gt);
  if (rc) return rc;
  ResetLaunch p;
  memset(&p, 0, sizeof p);
  p.st = e->st;
  p.games = e->games_d;
  p.images = e->images_d;
  p.groups = gt->dev;
  p.n_groups = gt->count;
  p.mask = mask_dev;
  p.obs = obs_dev;
  p.S = e->S;
  p.quirks = e->quirks;
  p.ipw = e->cfg.inst_per_warp;
  cudaError_t r = launch_reset(p, e->cfg.block, e->stream);
  return r == cudaSuccess ? OCTAX_OK : cuda_fail(r, "octax_reset");
}

int octax_step(octax_env *e, const uint8_t *actions_dev, uint8_t *obs_dev, float *reward_dev,
               uint8_t *done_dev) {
  if (!e) {
    set_error("octax_step: null env");
    return OCTAX_EINVAL;
  }
  int rc = check_io(actions_dev, obs_dev, reward_dev, done_dev);
  if (rc) return rc;
  IO io{actions_dev, obs_dev, reward_dev, done_dev, e->n};
  octax_launch cfg = e->cfg;
  cfg.steps_per_launch = 1;
  cfg.use_graph = 0;
  return enqueue_steps(e, cfg, 1, io);
}

int octax_step_n(octax_env *e, int n_steps, const uint8_t *actions_dev, uint8_t *obs_dev,
                 float *reward_dev, uint8_t *done_dev) {
  if (!e || n_steps < 1) {
    set_error("octax_step_n: need env and n_steps >= 1");
    return OCTAX_EINVAL;
  }
  int rc = check_io(actions_dev, obs_dev, reward_dev, done_dev);
  if (rc) return rc;
  IO io{actions_dev, obs_dev, reward_dev, done_dev, e->n};
  return enqueue_steps(e, e->cfg, n_steps, io);
}

int octax_step_n_packed(octax_env *e, int n_steps, const uint8_t *actions_dev, uint64_t *obs_words_dev,
                        float *reward_dev, uint8_t *done_dev) {
  if (!e || n_steps < 1) {
    set_error("octax_step_n_packed: need env and n_steps >= 1");
    return OCTAX_EINVAL;
  }
  uint8_t *obs = reinterpret_cast<uint8_t *>(obs_words_dev);
  int rc = check_io(actions_dev, obs, reward_dev, done_dev);
  if (rc) return rc;
  IO io{actions_dev, obs, reward_dev, done_dev, e->n, 1, 0};
  octax_launch cfg = e->cfg;
  cfg.writer_warps = 0;  // the writer warps write uint8 frames only
  return enqueue_steps(e, cfg, n_steps, io);
}

// Device-accessible address of a page-locked host buffer, or nullptr.
static void *mapped_host(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error of an unknown pointer
    return nullptr;
  }
  return (a.type == cudaMemoryTypeHost && a.devicePointer) ? a.devicePointer : nullptr;
}

namespace {

// One env step on device buffers, uint8 or packed frames (no graph).
int step_once(octax_env *e, const uint8_t *actions_dev, uint8_t *obs_dev, float *reward_dev, uint8_t *done_dev,
              int packed) {
  int rc = check_io(actions_dev, obs_dev, reward_dev, done_dev);
  if (rc) return rc;
  IO io{actions_dev, obs_dev, reward_dev, done_dev, e->n, packed, 0};
  octax_launch cfg = e->cfg;
  cfg.steps_per_launch = 1;
  cfg.use_graph = 0;
  if (packed) cfg.writer_warps = 0;
  return enqueue_steps(e, cfg, 1, io);
}

int step_host(octax_env *e, const uint8_t *actions_host, uint8_t *obs_host, float *reward_host,
              uint8_t *done_host, int packed, const char *who) {
  if (!e || !actions_host || !obs_host || !reward_host || !done_host) {
    set_error(std::string(who) + ": null argument");
    return OCTAX_EINVAL;
  }
  // Page-locked buffers are device-mapped: the kernel reads the actions and
  // streams observations, rewards and flags straight into them over the
  // host link, with no staging copy.
  void *d_act = mapped_host(actions_host), *d_obs = mapped_host(obs_host);
  void *d_rew = mapped_host(reward_host), *d_done = mapped_host(done_host);
  if (d_act && d_obs && d_rew && d_done && aligned16(d_obs)) {
    int rc = step_once(e, static_cast<const uint8_t *>(d_act), static_cast<uint8_t *>(d_obs),
                       static_cast<float *>(d_rew), static_cast<uint8_t *>(d_done), packed);
    if (rc) return rc;
    cudaError_t r = cudaStreamSynchronize(e->stream);
    return r == cudaSuccess ? OCTAX_OK : cuda_fail(r, who);
  }
  const size_t n = (size_t)e->n;
  const size_t obs_bytes = n * (size_t)e->S * (packed ? packed_frame_bytes(e->schip) : frame_bytes(e->schip));
  if (!e->hs_act) {  // staging sized for uint8 frames, which are the larger
    cudaError_t r = dalloc(e, &e->hs_act, n);
    if (r == cudaSuccess) r = dalloc(e, &e->hs_obs, n * (size_t)e->S * frame_bytes(e->schip));
    if (r == cudaSuccess) r = dalloc(e, &e->hs_rew, n);
    if (r == cudaSuccess) r = dalloc(e, &e->hs_done, n);
    if (r != cudaSuccess) {
      set_error(std::string(who) + ": staging allocation failed");
      return OCTAX_ENOMEM;
    }
  }
  cudaError_t r = cudaMemcpyAsync(e->hs_act, actions_host, n, cudaMemcpyHostToDevice, e->stream);
  if (r != cudaSuccess) return cuda_fail(r, who);
  int rc = step_once(e, e->hs_act, e->hs_obs, e->hs_rew, e->hs_done, packed);
  if (rc) return rc;
  r = cudaMemcpyAsync(obs_host, e->hs_obs, obs_bytes, cudaMemcpyDeviceToHost, e->stream);
  if (r == cudaSuccess) r = cudaMemcpyAsync(reward_host, e->hs_rew, n * 4, cudaMemcpyDeviceToHost, e->stream);
  if (r == cudaSuccess) r = cudaMemcpyAsync(done_host, e->hs_done, n, cudaMemcpyDeviceToHost, e->stream);
  if (r == cudaSuccess) r = cudaStreamSynchronize(e->stream);
  return r == cudaSuccess ? OCTAX_OK : cuda_fail(r, who);
}

}  // namespace

int octax_step_host(octax_env *e, const uint8_t *actions_host, uint8_t *obs_host, float *reward_host,
                    uint8_t *done_host) {
  return step_host(e, actions_host, obs_host, reward_host, done_host, 0, "octax_step_host");
}

int octax_step_host_packed(octax_env *e, const uint8_t *actions_host, uint64_t *obs_words_host,
                           float *reward_host, uint8_t *done_host) {
  return step_host(e, actions_host, reinterpret_cast<uint8_t *>(obs_words_host), reward_host, done_host, 1,
                   "octax_step_host_packed");
}

int octax_state_hash(octax_env *e, uint64_t *hash_dev) {
  if (!e || !hash_dev) {
    set_error("octax_state_hash: null argument");
    return OCTAX_EINVAL;
  }
  cudaError_t r = launch_hash(e->st, e->images_d, e->slot_of_row_d, e->n, hash_dev, e->stream);
  return r == cudaSuccess ? OCTAX_OK : cuda_fail(r, "octax_state_hash");
}

int octax_get_state(octax_env *e, int64_t first, int64_t count, octax_state_record *out_host) {
  if (!e || !out_host || first < 0 || count < 0 || first + count > e->n) {
    set_error("octax_get_state: range outside [0, n_envs) or null output");
    return OCTAX_EINVAL;
  }
  if (count == 0) return OCTAX_OK;
  octax_state_record *tmp = nullptr;
  cudaError_t r = cudaMallocAsync(&tmp, count * sizeof(octax_state_record), e->stream);
  if (r != cudaSuccess) return cuda_fail(r, "octax_get_state alloc");
  r = launch_records(e->st, e->images_d, e->slot_of_row_d, first, count, tmp, e->stream);
  if (r == cudaSuccess)
    r = cudaMemcpyAsync(out_host, tmp, count * sizeof(octax_state_record), cudaMemcpyDeviceToHost, e->stream);
  cudaFreeAsync(tmp, e->stream);
  if (r == cudaSuccess) r = cudaStreamSynchronize(e->stream);
  return r == cudaSuccess ? OCTAX_OK : cuda_fail(r, "octax_get_state");
}

int octax_set_state(octax_env *e, int64_t first, int64_t count, const octax_state_record *in_host) {
  if (!e || !in_host || first < 0 || count < 0 || first + count > e->n) {
    set_error("octax_set_state: range outside [0, n_envs) or null input");
    return OCTAX_EINVAL;
  }
  for (int64_t i = 0; i < count; ++i)
    if (in_host[i].SP > 16) {
      set_error("octax_set_state: SP > 16");
      return OCTAX_EINVAL;
    }
  if (count == 0) return OCTAX_OK;
  octax_state_record *tmp = nullptr;
  cudaError_t r = cudaMallocAsync(&tmp, count * sizeof(octax_state_record), e->stream);
  if (r != cudaSuccess) return cuda_fail(r, "octax_set_state alloc");
  r = cudaMemcpyAsync(tmp, in_host, count * sizeof(octax_state_record), cudaMemcpyHostToDevice, e->stream);
  if (r == cudaSuccess)
    r = launch_set_records(e->st, e->games_d, e->images_d, e->slot_of_row_d, first, count, tmp, e->stream);
  cudaFreeAsync(tmp, e->stream);
  if (r == cudaSuccess) r = cudaStreamSynchronize(e->stream);
  return r == cudaSuccess ? OCTAX_OK : cuda_fail(r, "octax_set_state");
}

int octax_sync(octax_env *e, int timeout_ms) {
  if (!e) {
    set_error("octax_sync: null env");
    return OCTAX_EINVAL;
  }
  cudaError_t r = cudaEventRecord(e->ev, e->stream);
  if (r != cudaSuccess) return cuda_fail(r, "octax_sync record");
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    r = cudaEventQuery(e->ev);
    if (r == cudaSuccess) {
      unsigned int err = 0;
      r = cudaMemcpy(&err, e->err_d, sizeof err, cudaMemcpyDeviceToHost);
      if (r != cudaSuccess) return cuda_fail(r, "octax_sync");
      if (err) {
        r = cudaMemsetAsync(e->err_d, 0, sizeof(unsigned int), e->stream);
        if (r == cudaSuccess) r = cudaStreamSynchronize(e->stream);
        if (r != cudaSuccess) return cuda_fail(r, "octax_sync");
        set_error("octax_sync: a kernel's shared-memory hand-over timed out; outputs are incomplete");
        return OCTAX_ECUDA;
      }
      return OCTAX_OK;
    }
    if (r != cudaErrorNotReady) return cuda_fail(r, "octax_sync");
    if (timeout_ms >= 0 &&
        std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms)) {
      set_error("octax_sync: timed out");
      return OCTAX_ETIMEOUT;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

int octax_debug_stall_writers(octax_env *e, int on) {
  if (!e) {
    set_error("octax_debug_stall_writers: null env");
    return OCTAX_EINVAL;
  }
  cudaError_t r = cudaStreamSynchronize(e->stream);
  if (r != cudaSuccess) return cuda_fail(r, "octax_debug_stall_writers");
  for (auto &kv : e->graphs) cudaGraphExecDestroy(kv.second);
  e->graphs.clear();
  e->stall_writers = on ? 1 : 0;
  return OCTAX_OK;
}

int octax_get_launch(const octax_env *e, octax_launch *out) {
  if (!e || !out) {
    set_error("octax_get_launch: null argument");
    return OCTAX_EINVAL;
  }
  *out = e->cfg;
  return OCTAX_OK;
}

int octax_set_launch(octax_env *e, const octax_launch *cfg) {
  if (!e || !cfg) {
    set_error("octax_set_launch: null argument");
    return OCTAX_EINVAL;
  }
  if (const char *why = launch_problem(*cfg, e->schip)) {
    set_error(std::string("octax_set_launch: ") + why);
    return OCTAX_EINVAL;
  }
  e->cfg = *cfg;
  return OCTAX_OK;
}

int octax_autotune(octax_env *e, int n_steps, const uint8_t *actions_dev, float *best_ms_out) {
  if (!e || n_steps < 1) {
    set_error("octax_autotune: need env and n_steps >= 1");
    return OCTAX_EINVAL;
  }
  const size_t n = (size_t)e->n;
  // back up the mutable state so that tuning leaves no trace
  const DevState &st = e->st;
  struct Piece {
    void *p;
    size_t bytes;
  };
  const Piece pieces[] = {{st.v, 16 * n},     {st.pcI, 4 * n},    {st.misc, 4 * n},
                          {st.stack, 32 * n}, {st.disp, 8 * (size_t)disp_words(e->schip) * n}, {st.dirty, 8 * n},
                          {st.ram, 4096 * n}, {st.ep, 4 * n},     {st.env_steps, 4 * n},
                          {st.prev_score, 4 * n}, {st.last_act, n}, {st.mode, n}, {st.rpl, 16 * n},
                          {st.wrange, 4 * n}};
  size_t total = 0;
  for (const Piece &pc : pieces) total += pc.bytes;
  uint8_t *backup = nullptr, *acts = nullptr, *obs = nullptr, *done = nullptr;
  float *rew = nullptr;
  const size_t obs_bytes = (size_t)n_steps * n * e->S * frame_bytes(e->schip);
  cudaError_t r = cudaMalloc(&backup, total);
  if (r == cudaSuccess) r = cudaMalloc(&acts, (size_t)n_steps * n);
  if (r == cudaSuccess) r = cudaMalloc(&obs, obs_bytes);
  if (r == cudaSuccess) r = cudaMalloc((void **)&rew, (size_t)n_steps * n * 4);
  if (r == cudaSuccess) r = cudaMalloc(&done, (size_t)n_steps * n);
  if (r != cudaSuccess) {
    cudaFree(backup);
    cudaFree(acts);
    cudaFree(obs);
    cudaFree(rew);
    cudaFree(done);
    set_error("octax_autotune: scratch allocation failed");
    return OCTAX_ENOMEM;
  }
  // copy the state pieces to (save) or from (restore) the backup
  auto copy_state = [&](bool save) {
    size_t off = 0;
    cudaError_t err = cudaSuccess;
    for (const Piece &pc : pieces) {
      const cudaError_t c =
          save ? cudaMemcpyAsync(backup + off, pc.p, pc.bytes, cudaMemcpyDeviceToDevice, e->stream)
               : cudaMemcpyAsync(pc.p, backup + off, pc.bytes, cudaMemcpyDeviceToDevice, e->stream);
      if (err == cudaSuccess) err = c;
      off += pc.bytes;
    }
    return err;
  };
  r = copy_state(true);
  if (r == cudaSuccess && actions_dev) {
    r = cudaMemcpyAsync(acts, actions_dev, (size_t)n_steps * n, cudaMemcpyDeviceToDevice, e->stream);
  } else if (r == cudaSuccess) {  // uniform over each game's action indices (including the no-op)
    std::vector<uint8_t> h((size_t)n_steps * n);
    uint64_t x = 0x9E3779B97F4A7C15ull;
    for (size_t i = 0; i < h.size(); ++i) {
      x += 0x9E3779B97F4A7C15ull;  // splitmix64
      uint64_t z = x;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      h[i] = (uint8_t)(z % 5u);
    }
    r = cudaMemcpyAsync(acts, h.data(), h.size(), cudaMemcpyHostToDevice, e->stream);
    if (r == cudaSuccess) r = cudaStreamSynchronize(e->stream);  // h is a local buffer
  }
  IO io{acts, obs, rew, done, e->n};
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (r == cudaSuccess) r = cudaEventCreate(&t0);
  if (r == cudaSuccess) r = cudaEventCreate(&t1);
  const octax_launch saved = e->cfg;
  octax_launch best = saved;
  float best_ms = 1e30f;
  int rc = r == cudaSuccess ? OCTAX_OK : cuda_fail(r, "octax_autotune setup");
  // Every candidate runs the same n_steps from the caller's state (restored
  // before the warm-up and before each timed repetition), so all of them
  // see the same phase of the workload (episode ends, resets).
  auto trial = [&](const octax_launch &c) {
    if (rc != OCTAX_OK || launch_problem(c, e->schip) || c.steps_per_launch > n_steps) return;
    e->cfg = c;
    cudaError_t q = copy_state(false);
    rc = q == cudaSuccess ? enqueue_steps(e, c, n_steps, io) : cuda_fail(q, "octax_autotune");  // warm-up
    float ms_min = 1e30f;
    for (int rep = 0; rep < 3 && rc == OCTAX_OK; ++rep) {
      q = copy_state(false);
      if (q == cudaSuccess) q = cudaEventRecord(t0, e->stream);
      if (q != cudaSuccess) {
        rc = cuda_fail(q, "octax_autotune");
        break;
      }
      rc = enqueue_steps(e, c, n_steps, io);
      q = cudaEventRecord(t1, e->stream);
      if (q == cudaSuccess) q = cudaEventSynchronize(t1);
      float ms = 0;
      if (q == cudaSuccess) q = cudaEventElapsedTime(&ms, t0, t1);
      if (q != cudaSuccess && rc == OCTAX_OK) rc = cuda_fail(q, "octax_autotune");
      ms_min = std::min(ms_min, ms);
    }
    if (rc == OCTAX_OK && ms_min < best_ms) {
      best_ms = ms_min;
      best = c;
    }
  };
  // stage 1: CTA shape (threads x instances per warp) and balanced waves,
  // plain kernel, up to 32 steps per launch (long launches rank shapes as
  // they will run)
  for (int b : {32, 64, 128, 256})
    for (int ipw : {32, 16, 8, 7, 6, 4})
      for (int bal : {0, 1}) {
        const int J = b / 32 * ipw;
        if (J >= 8 && J <= 256) trial(octax_launch{b, ipw, std::min(32, n_steps), 0, 1, 0, bal});
      }
  // stage 2: writer warps, persistence and steps per launch around the best
  // shape. Launches up to 256 steps and the call length itself are
  // candidates: a launch ends with its slowest warp, and on workloads whose
  // instances now and then run a long sequential stretch (no-op resets) the
  // longer launch spreads that wait over more steps.
  const octax_launch shape = best;
  std::vector<int> spls = {1, 2, 4, 8, 16, 32, 64, 128, 256};
  if (n_steps <= 256 && std::find(spls.begin(), spls.end(), n_steps) == spls.end()) spls.push_back(n_steps);
  for (int W : {0, 1, 2, 4})
    for (int pers : {0, 1})
      for (int spl : spls)
        trial(octax_launch{shape.block, shape.inst_per_warp, spl, pers, 1, W, shape.balance});
  r = copy_state(false);
  const cudaError_t rs = cudaStreamSynchronize(e->stream);
  if (r == cudaSuccess) r = rs;
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaFree(backup);
  cudaFree(acts);
  cudaFree(obs);
  cudaFree(rew);
  cudaFree(done);
  if (rc) {
    e->cfg = saved;
    return rc;
  }
  if (r != cudaSuccess) {
    e->cfg = saved;
    return cuda_fail(r, "octax_autotune");
  }
  e->cfg = best;
  if (best_ms_out) *best_ms_out = best_ms;
  return OCTAX_OK;
}

int64_t octax_num_envs(const octax_env *e) { return e ? e->n : -1; }
int octax_stack_frames(const octax_env *e) { return e ? e->S : -1; }
int octax_variant(const octax_env *e) {
  return e ? (e->schip ? (int)OCTAX_VARIANT_SCHIP : (int)OCTAX_VARIANT_CHIP8) : -1;
}
size_t octax_device_bytes(const octax_env *e) { return e ? e->bytes : 0; }

void octax_destroy(octax_env *e) { free_env(e); }

}  // extern "C"
