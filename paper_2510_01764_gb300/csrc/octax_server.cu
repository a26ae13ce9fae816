// liboctax serving loop: continuous batching of environment-step requests.
//
// One server thread owns a CUDA stream and a pool of resident emulator slots
// sized by a device-memory budget. Requests (game, n_envs, n_steps, actions,
// seed, caller-owned output buffers) queue on submission; at every tick the
// thread admits queued requests whose instances fit in the free slots (reset
// kernel into those slots), then launches ONE step kernel over the groups of
// every running request, each group writing into its own request's buffers
// at that request's current step. Requests join and leave between ticks, so
// new arrivals ride along with work already on the GPU; a request's slots are
// recycled as soon as its last tick is enqueued (stream order makes that safe)
// and it is reported done when that tick's event completes.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "octax_internal.h"

using namespace octax;

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Req {
  uint64_t id;
  octax_request r;
  std::vector<uint8_t> actions;  // host copy [n_steps][n_envs]
  int64_t submit_ns = 0, admit_ns = 0, done_ns = 0;
  int state = 0;                 // 0 queued, 1 running, 2 done
  uint32_t slot0 = 0;
  uint32_t steps_done = 0;
};

// First-fit allocator of contiguous slot ranges.
struct RangeAlloc {
  std::map<uint32_t, uint32_t> free_;  // start -> length
  uint32_t used = 0;
  explicit RangeAlloc(uint32_t cap) {
    if (cap) free_[0] = cap;
  }
  bool alloc(uint32_t n, uint32_t *out) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *out = it->first;
        const uint32_t start = it->first + n, len = it->second - n;
        free_.erase(it);
        if (len) free_[start] = len;
        used += n;
        return true;
      }
    }
    return false;
  }
  void release(uint32_t start, uint32_t n) {
    used -= n;
    auto it = free_.emplace(start, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

// Pinned host + device table pair for one in-flight tick.
struct TickBuf {
  Group *h_groups = nullptr, *d_groups = nullptr;
  IO *h_io = nullptr, *d_io = nullptr;
  uint64_t *h_seeds = nullptr, *d_seeds = nullptr;
  Group *h_rgroups = nullptr, *d_rgroups = nullptr;  // reset groups of admissions
  size_t cap_groups = 0, cap_io = 0;
  cudaEvent_t ev = nullptr;
  bool pending = false;
  std::vector<uint64_t> completing;  // requests whose last step is in this tick
};

constexpr uint32_t kMaxEnvs = 4096;
constexpr uint32_t kMaxSteps = 8;

}  // namespace

struct octax_server {
  int device = 0;
  cudaStream_t stream = nullptr;
  int block = 64;   // threads per CTA
  int ipw = 8;      // instances per warp
  int J = 16;       // instances per CTA
  int depth = 2;
  int n_games = 0, S = 4;
  int schip = 0;  // OCTAX_VARIANT_SCHIP games
  uint32_t quirks = 0;
  uint32_t capacity = 0;
  std::vector<GameDev> games_h;
  GameDev *games_d = nullptr;
  uint8_t *images_d = nullptr;
  DevState st{};
  void *state_block = nullptr;
  uint8_t *act_arena = nullptr;  // [capacity * kMaxSteps]
  unsigned int *err_d = nullptr;
  RangeAlloc slots{0};
  std::vector<TickBuf> ticks;
  int64_t tick_no = 0;

  std::mutex mu;
  std::condition_variable cv_submit, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Req> reqs;
  std::vector<uint64_t> running;
  uint64_t next_id = 1;
  bool stop = false;
  std::string fatal;
  octax_server_stats stats{};
  std::thread th;
};

namespace {

int grow_tick(octax_server *s, TickBuf &t, size_t groups, size_t ios) {
  if (groups <= t.cap_groups && ios <= t.cap_io) return OCTAX_OK;
  cudaStreamSynchronize(s->stream);  // no tick may still read the old tables
  const size_t g = std::max(groups, 2 * t.cap_groups) + 64, io = std::max(ios, 2 * t.cap_io) + 16;
  cudaFreeHost(t.h_groups);
  cudaFreeHost(t.h_io);
  cudaFreeHost(t.h_seeds);
  cudaFreeHost(t.h_rgroups);
  cudaFree(t.d_groups);
  cudaFree(t.d_io);
  cudaFree(t.d_seeds);
  cudaFree(t.d_rgroups);
  cudaError_t r = cudaMallocHost(&t.h_groups, g * sizeof(Group));
  if (r == cudaSuccess) r = cudaMallocHost(&t.h_rgroups, g * sizeof(Group));
  if (r == cudaSuccess) r = cudaMallocHost(&t.h_seeds, g * sizeof(uint64_t));
  if (r == cudaSuccess) r = cudaMallocHost(&t.h_io, io * sizeof(IO));
  if (r == cudaSuccess) r = cudaMalloc(&t.d_groups, g * sizeof(Group));
  if (r == cudaSuccess) r = cudaMalloc(&t.d_rgroups, g * sizeof(Group));
  if (r == cudaSuccess) r = cudaMalloc(&t.d_seeds, g * sizeof(uint64_t));
  if (r == cudaSuccess) r = cudaMalloc(&t.d_io, io * sizeof(IO));
  if (r != cudaSuccess) return cuda_fail(r, "server tick tables");
  t.cap_groups = g;
  t.cap_io = io;
  return OCTAX_OK;
}

void finish_tick(octax_server *s, TickBuf &t) {
  const int64_t now = now_ns();
  std::lock_guard<std::mutex> lk(s->mu);
  for (uint64_t id : t.completing) {
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) continue;
    it->second.state = 2;
    it->second.done_ns = now;
    s->stats.completed++;
  }
  t.completing.clear();
  t.pending = false;
  s->cv_done.notify_all();
}

// One scheduling round: admit, then launch one batched step kernel over all
// running requests, advancing each by the fewest steps any of them has left
// (so that none runs past its last step). Returns false when there was
// nothing to launch.
bool tick(octax_server *s) {
  TickBuf &t = s->ticks[s->tick_no % s->depth];
  if (t.pending) {  // ring slot still in flight: wait for it
    cudaEventSynchronize(t.ev);
    finish_tick(s, t);
  }
  std::vector<Req *> admitted, run;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    // FIFO admission while the head fits
    while (!s->queue.empty()) {
      Req &q = s->reqs[s->queue.front()];
      uint32_t slot0;
      if (!s->slots.alloc(q.r.n_envs, &slot0)) break;
      q.slot0 = slot0;
      q.state = 1;
      q.admit_ns = now_ns();
      s->queue.pop_front();
      s->running.push_back(q.id);
      admitted.push_back(&q);
    }
    for (uint64_t id : s->running) run.push_back(&s->reqs[id]);
  }
  if (run.empty()) return false;
  uint32_t k_steps = kMaxSteps;  // steps of this tick
  for (Req *q : run) k_steps = std::min<uint32_t>(k_steps, q->r.n_steps - q->steps_done);
  const int B = s->J;  // instances per CTA
  size_t n_groups = 0, n_rgroups = 0;
  for (Req *q : run) n_groups += (q->r.n_envs + B - 1) / B;
  for (Req *q : admitted) n_rgroups += (q->r.n_envs + B - 1) / B;
  if (grow_tick(s, t, std::max(n_groups, n_rgroups), run.size())) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->fatal = "server tick: table allocation failed";
    s->stop = true;
    s->cv_done.notify_all();
    return false;
  }
  cudaError_t r = cudaSuccess;
  // ---- admissions: actions into the arena, reset the slots
  if (!admitted.empty()) {
    size_t k = 0;
    for (Req *q : admitted) {
      r = cudaMemcpyAsync(s->act_arena + (size_t)q->slot0 * kMaxSteps, q->actions.data(),
                          q->actions.size(), cudaMemcpyHostToDevice, s->stream);
      for (uint32_t c = 0; c < q->r.n_envs; c += B) {
        t.h_rgroups[k] = Group{q->slot0 + c, (uint16_t)std::min<uint32_t>(B, q->r.n_envs - c), q->r.game, 0u, c};
        t.h_seeds[k] = q->r.seed;
        ++k;
      }
    }
    if (r == cudaSuccess) r = cudaMemcpyAsync(t.d_rgroups, t.h_rgroups, k * sizeof(Group), cudaMemcpyHostToDevice, s->stream);
    if (r == cudaSuccess) r = cudaMemcpyAsync(t.d_seeds, t.h_seeds, k * sizeof(uint64_t), cudaMemcpyHostToDevice, s->stream);
    ResetLaunch p;
    memset(&p, 0, sizeof p);
    p.st = s->st;
    p.games = s->games_d;
    p.images = s->images_d;
    p.groups = t.d_rgroups;
    p.n_groups = (int)k;
    p.S = s->S;
    p.quirks = s->quirks;
    p.ipw = s->ipw;
    p.init = 1;
    p.seed_of_group = t.d_seeds;
    p.set_rows = 1;
    if (r == cudaSuccess) r = launch_reset(p, s->block, s->stream);
  }
  // ---- one batched step over every running request
  size_t g = 0;
  for (size_t i = 0; i < run.size(); ++i) {
    Req *q = run[i];
    const size_t n = q->r.n_envs, st = q->steps_done;
    t.h_io[i] = IO{s->act_arena + (size_t)q->slot0 * kMaxSteps + st * n,
                   q->r.obs_dev + st * n * (size_t)s->S * frame_bytes(s->schip), q->r.reward_dev + st * n,
                   q->r.done_dev + st * n, (int64_t)n};
    for (uint32_t c = 0; c < q->r.n_envs; c += B)
      t.h_groups[g++] = Group{q->slot0 + c, (uint16_t)std::min<uint32_t>(B, q->r.n_envs - c), q->r.game,
                              (uint32_t)i, c};
  }
  if (r == cudaSuccess) r = cudaMemcpyAsync(t.d_groups, t.h_groups, g * sizeof(Group), cudaMemcpyHostToDevice, s->stream);
  if (r == cudaSuccess) r = cudaMemcpyAsync(t.d_io, t.h_io, run.size() * sizeof(IO), cudaMemcpyHostToDevice, s->stream);
  StepLaunch p;
  memset(&p, 0, sizeof p);
  p.st = s->st;
  p.games = s->games_d;
  p.images = s->images_d;
  p.groups = t.d_groups;
  p.n_groups = (int)g;
  p.io_table = t.d_io;
  p.step0 = 0;
  p.steps = (int)k_steps;
  p.S = s->S;
  p.quirks = s->quirks;
  p.ipw = s->ipw;
  p.err = s->err_d;
  p.wrappers = uses_wrappers(s->games_h.data(), s->games_h.size());
  if (r == cudaSuccess) r = launch_step(p, (int)g, s->block, s->stream);
  if (r == cudaSuccess) r = cudaEventRecord(t.ev, s->stream);
  if (r != cudaSuccess) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->fatal = std::string("server tick: ") + cudaGetErrorString(r);
    s->stop = true;
    s->cv_done.notify_all();
    return false;
  }
  t.pending = true;
  // ---- advance; requests whose last step was enqueued give their slots back
  {
    std::lock_guard<std::mutex> lk(s->mu);
    int64_t envs = 0;
    std::vector<uint64_t> still;
    for (Req *q : run) {
      q->steps_done += k_steps;
      envs += q->r.n_envs;
      if (q->steps_done == q->r.n_steps) {
        t.completing.push_back(q->id);
        s->slots.release(q->slot0, q->r.n_envs);
      } else {
        still.push_back(q->id);
      }
    }
    s->running.swap(still);
    s->stats.ticks++;
    s->stats.env_steps += envs * (int64_t)k_steps;
    s->stats.peak_active_envs = std::max(s->stats.peak_active_envs, envs);
    s->stats.peak_active_requests = std::max<int64_t>(s->stats.peak_active_requests, (int64_t)run.size());
  }
  s->tick_no++;
  return true;
}

void loop(octax_server *s) {
  cudaSetDevice(s->device);
  for (;;) {
    // retire finished ticks (oldest first)
    for (int k = 0; k < s->depth; ++k) {
      TickBuf &t = s->ticks[(s->tick_no + k) % s->depth];
      if (t.pending && cudaEventQuery(t.ev) == cudaSuccess) finish_tick(s, t);
    }
    bool launched = tick(s);
    if (!launched) {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop) break;
      bool inflight = false;
      for (auto &t : s->ticks) inflight |= t.pending;
      if (s->queue.empty() && s->running.empty() && !inflight)
        s->cv_submit.wait_for(lk, std::chrono::milliseconds(5));
      else if (s->running.empty())
        lk.unlock(), std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->stop) break;
    }
  }
  cudaStreamSynchronize(s->stream);
  for (auto &t : s->ticks)
    if (t.pending) finish_tick(s, t);
}

}  // namespace

extern "C" {

int octax_server_create(const octax_game *games, int n_games, uint32_t quirks,
                        const octax_server_config *cfg, octax_server **out) {
  if (!out || !games || !cfg || n_games < 1 || n_games > 65535 || (quirks & ~0x3Fu)) {
    set_error("octax_server_create: need out, games, cfg, 1..65535 games, known quirks");
    return OCTAX_EINVAL;
  }
  *out = nullptr;
  const int B = cfg->block ? cfg->block : 64;
  const int ipw = cfg->inst_per_warp ? cfg->inst_per_warp : 8;
  const int depth = cfg->max_inflight_ticks ? cfg->max_inflight_ticks : 2;
  if (!(B == 32 || B == 64 || B == 128 || B == 256) || depth < 1 || depth > 8 ||
      !(ipw == 1 || ipw == 2 || ipw == 4 || ipw == 8 || ipw == 16 || ipw == 32)) {
    set_error("octax_server_create: block in {32,64,128,256}, inst_per_warp in {1..32}, "
              "max_inflight_ticks 1..8");
    return OCTAX_EINVAL;
  }
  const int schip = games[0].variant == OCTAX_VARIANT_SCHIP;
  if (step_smem_bytes(B, ipw, schip) > max_dynamic_smem()) {
    set_error("octax_server_create: too many instances per CTA for shared memory");
    return OCTAX_EINVAL;
  }
  const int64_t per_slot = (int64_t)(slot_state_bytes(schip) + kMaxSteps);
  const int64_t cap64 = cfg->memory_budget_bytes / per_slot;
  if (cap64 < 1 || cap64 > ((int64_t)1 << 31)) {
    set_error("octax_server_create: memory budget must hold 1 .. 2^31 instances");
    return OCTAX_EINVAL;
  }
  std::vector<GameDev> games_dev;
  std::vector<uint8_t> images;
  {
    int rc = build_games(games, n_games, games_dev, images);
    if (rc) return rc;
  }
  octax_server *s = new octax_server();
  cudaGetDevice(&s->device);
  s->block = B;
  s->ipw = ipw;
  s->J = B / 32 * ipw;
  s->depth = depth;
  s->n_games = n_games;
  s->S = games[0].stack_frames;
  s->schip = schip;
  s->quirks = quirks;
  s->capacity = (uint32_t)cap64;
  s->slots = RangeAlloc(s->capacity);
  s->games_h = games_dev;
  size_t bytes = 0;
  cudaError_t r = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (r == cudaSuccess) r = alloc_state(s->st, s->capacity, s->schip, &s->state_block, &bytes);
  if (r == cudaSuccess) r = cudaMalloc(&s->act_arena, (size_t)s->capacity * kMaxSteps);
  if (r == cudaSuccess) r = cudaMalloc(&s->err_d, sizeof(unsigned int));
  if (r == cudaSuccess) r = cudaMemset(s->err_d, 0, sizeof(unsigned int));
  if (r == cudaSuccess) r = cudaMalloc(&s->games_d, s->games_h.size() * sizeof(GameDev));
  if (r == cudaSuccess) r = cudaMalloc(&s->images_d, images.size());
  if (r == cudaSuccess)
    r = cudaMemcpy(s->games_d, s->games_h.data(), s->games_h.size() * sizeof(GameDev), cudaMemcpyHostToDevice);
  if (r == cudaSuccess) r = cudaMemcpy(s->images_d, images.data(), images.size(), cudaMemcpyHostToDevice);
  s->ticks.resize(depth);
  for (auto &t : s->ticks)
    if (r == cudaSuccess) r = cudaEventCreateWithFlags(&t.ev, cudaEventDisableTiming);
  if (r != cudaSuccess) {
    int rc = r == cudaErrorMemoryAllocation ? OCTAX_ENOMEM : cuda_fail(r, "octax_server_create");
    if (rc == OCTAX_ENOMEM) set_error("octax_server_create: device allocation failed");
    octax_server_destroy(s);
    return rc;
  }
  s->stats.slots_capacity = s->capacity;
  s->th = std::thread(loop, s);
  *out = s;
  return OCTAX_OK;
}

static int check_request(const octax_server *s, const octax_request &r, const char *who) {
  if (r.game >= s->n_games || r.n_envs < 1 || r.n_envs > kMaxEnvs || r.n_steps < 1 ||
      r.n_steps > kMaxSteps || !r.actions_host || !r.obs_dev || !r.reward_dev || !r.done_dev ||
      (reinterpret_cast<uintptr_t>(r.obs_dev) & 15u)) {
    set_error(std::string(who) + ": need game < n_games, 1..4096 envs, 1..8 steps, all buffers, "
                                 "16-byte aligned obs");
    return OCTAX_EINVAL;
  }
  if (r.n_envs > s->capacity) {
    set_error(std::string(who) + ": request larger than the memory budget admits");
    return OCTAX_ENOMEM;
  }
  return OCTAX_OK;
}

// Queue already checked requests (caller holds s->mu).
static void enqueue_locked(octax_server *s, const octax_request *reqs, int n, uint64_t *ids) {
  const int64_t t = now_ns();
  for (int k = 0; k < n; ++k) {
    const octax_request &r = reqs[k];
    const uint64_t id = s->next_id++;
    Req &q = s->reqs[id];
    q.id = id;
    q.r = r;
    q.actions.assign(r.actions_host, r.actions_host + (size_t)r.n_steps * r.n_envs);
    q.r.actions_host = nullptr;
    q.submit_ns = t;
    s->queue.push_back(id);
    s->stats.submitted++;
    ids[k] = id;
  }
  s->cv_submit.notify_one();
}

int octax_server_submit(octax_server *s, const octax_request *req, uint64_t *id_out) {
  return octax_server_submit_batch(s, req, 1, id_out);
}

int octax_server_submit_batch(octax_server *s, const octax_request *reqs, int n, uint64_t *ids_out) {
  if (!s || !reqs || !ids_out || n < 1) {
    set_error("octax_server_submit: null argument or n < 1");
    return OCTAX_EINVAL;
  }
  for (int k = 0; k < n; ++k) {
    const int rc = check_request(s, reqs[k], "octax_server_submit");
    if (rc) return rc;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    set_error(s->fatal.empty() ? "octax_server_submit: server stopped" : s->fatal);
    return OCTAX_ECUDA;
  }
  enqueue_locked(s, reqs, n, ids_out);
  return OCTAX_OK;
}

static void fill_info(const Req &q, octax_request_info *out) {
  if (!out) return;
  out->state = q.state;
  out->submit_ns = q.submit_ns;
  out->admit_ns = q.admit_ns;
  out->done_ns = q.done_ns;
}

int octax_server_wait(octax_server *s, uint64_t id, int timeout_ms, octax_request_info *info_out) {
  if (!s) {
    set_error("octax_server_wait: null server");
    return OCTAX_EINVAL;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) {
    set_error("octax_server_wait: unknown request id");
    return OCTAX_ENOTFOUND;
  }
  auto ready = [&] { return s->reqs[id].state == 2 || s->stop; };
  if (timeout_ms < 0)
    s->cv_done.wait(lk, ready);
  else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    fill_info(s->reqs[id], info_out);
    set_error("octax_server_wait: timed out");
    return OCTAX_ETIMEOUT;
  }
  fill_info(s->reqs[id], info_out);
  if (s->reqs[id].state != 2) {
    set_error(s->fatal.empty() ? "octax_server_wait: server stopped" : s->fatal);
    return OCTAX_ECUDA;
  }
  return OCTAX_OK;
}

int octax_server_wait_batch(octax_server *s, const uint64_t *ids, int n, int timeout_ms, octax_request_info *infos,
                            int release) {
  if (!s || !ids || n < 1) {
    set_error("octax_server_wait_batch: null argument or n < 1");
    return OCTAX_EINVAL;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  for (int k = 0; k < n; ++k)
    if (s->reqs.find(ids[k]) == s->reqs.end()) {
      set_error("octax_server_wait_batch: unknown request id");
      return OCTAX_ENOTFOUND;
    }
  auto all_done = [&] {
    if (s->stop) return true;
    for (int k = 0; k < n; ++k)
      if (s->reqs[ids[k]].state != 2) return false;
    return true;
  };
  if (timeout_ms < 0)
    s->cv_done.wait(lk, all_done);
  else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), all_done)) {
    set_error("octax_server_wait_batch: timed out");
    return OCTAX_ETIMEOUT;
  }
  for (int k = 0; k < n; ++k)
    if (s->reqs[ids[k]].state != 2) {
      set_error(s->fatal.empty() ? "octax_server_wait_batch: server stopped" : s->fatal);
      return OCTAX_ECUDA;
    }
  for (int k = 0; k < n; ++k) {
    if (infos) fill_info(s->reqs[ids[k]], infos + k);
    if (release) s->reqs.erase(ids[k]);
  }
  return OCTAX_OK;
}

int octax_server_query(octax_server *s, uint64_t id, octax_request_info *info_out) {
  if (!s || !info_out) {
    set_error("octax_server_query: null argument");
    return OCTAX_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) {
    set_error("octax_server_query: unknown request id");
    return OCTAX_ENOTFOUND;
  }
  fill_info(it->second, info_out);
  return OCTAX_OK;
}

int octax_server_release(octax_server *s, uint64_t id) {
  if (!s) {
    set_error("octax_server_release: null server");
    return OCTAX_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) {
    set_error("octax_server_release: unknown request id");
    return OCTAX_ENOTFOUND;
  }
  if (it->second.state != 2) {
    set_error("octax_server_release: request not finished");
    return OCTAX_EINVAL;
  }
  s->reqs.erase(it);
  return OCTAX_OK;
}

int octax_server_get_stats(octax_server *s, octax_server_stats *out) {
  if (!s || !out) {
    set_error("octax_server_get_stats: null argument");
    return OCTAX_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->queued = (int64_t)s->queue.size();
  out->slots_in_use = s->slots.used;
  return OCTAX_OK;
}

void octax_server_destroy(octax_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_submit.notify_all();
  }
  if (s->th.joinable()) s->th.join();
  cudaSetDevice(s->device);
  for (auto &t : s->ticks) {
    cudaFreeHost(t.h_groups);
    cudaFreeHost(t.h_io);
    cudaFreeHost(t.h_seeds);
    cudaFreeHost(t.h_rgroups);
    cudaFree(t.d_groups);
    cudaFree(t.d_io);
    cudaFree(t.d_seeds);
    cudaFree(t.d_rgroups);
    if (t.ev) cudaEventDestroy(t.ev);
  }
  cudaFree(s->state_block);
  cudaFree(s->act_arena);
  cudaFree(s->err_d);
  cudaFree(s->games_d);
  cudaFree(s->images_d);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

}  // extern "C"
