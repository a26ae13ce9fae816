// octax_rollout_static: the environment step for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside another
// framework's memory pool or a pre-reserved arena, plugins whose host
// forbids allocation after start-up, and real-time loops where an
// allocation (which may synchronise the device) would break the timing
// budget. For them this file keeps everything the kernels need besides the
// caller's inputs and outputs -- the emulator state of up to
// kStaticMaxEnvs instances, the game descriptor, its 4 KB RAM image and the
// CTA group table -- in one file-scope __device__ array. Each loaded device
// holds that array (about 4.6 MB) until the process exits.
//
// The array's name is only a host-side stand-in in host code; the device
// address comes from cudaGetSymbolAddress, called once per device (with that
// device current) by the first call on it.
#include <cstring>
#include <mutex>
#include <vector>

#include "octax_internal.h"

namespace octax {
namespace {

constexpr int64_t kStaticMaxEnvs = 1024;
constexpr int kStaticBlock = 64;  // threads per CTA
constexpr int kStaticIpw = 16;    // instances per warp -> 32 instances per CTA
constexpr int kStaticPerCta = kStaticBlock / 32 * kStaticIpw;
constexpr int kStaticMaxGroups = (int)((kStaticMaxEnvs + kStaticPerCta - 1) / kStaticPerCta);

constexpr size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t N = (size_t)kStaticMaxEnvs;
// per-slot arrays, in the order of the pointer list in octax_rollout_static
constexpr size_t kArr[18] = {16 * N, 4 * N, 4 * N, 32 * N, 256 * N, 8 * N, 4096 * N,
                             4 * N,  4 * N, 4 * N, 8 * N,  4 * N,   4 * N, 2 * N, N, N, 16 * N, 4 * N};
constexpr size_t state_bytes() {
  size_t t = 0;
  for (size_t b : kArr) t += up256(b);
  return t;
}
constexpr size_t kOffGame = state_bytes();
constexpr size_t kOffImage = kOffGame + up256(sizeof(GameDev));
constexpr size_t kOffGroups = kOffImage + kRamBytes;
constexpr size_t kScratchBytes = kOffGroups + up256(kStaticMaxGroups * sizeof(Group));

static __device__ __align__(256) uint8_t g_scratch[kScratchBytes];

// Fills the descriptor, one half of the RAM image and the group table.
// Kernel parameters carry the host data, so no copy API is needed.
struct SetupArgs {
  GameDev game;
  uint8_t image_half[kRamBytes / 2];
  int half;
  int n_groups;
  uint32_t n_envs;
};

__global__ void static_setup_kernel(const SetupArgs a) {
  uint8_t *img = g_scratch + kOffImage + a.half * (kRamBytes / 2);
  for (int i = threadIdx.x; i < kRamBytes / 2; i += blockDim.x) img[i] = a.image_half[i];
  if (a.half != 0) return;
  if (threadIdx.x == 0) *reinterpret_cast<GameDev *>(g_scratch + kOffGame) = a.game;
  Group *groups = reinterpret_cast<Group *>(g_scratch + kOffGroups);
  for (int gi = threadIdx.x; gi < a.n_groups; gi += blockDim.x) {
    const uint32_t s0 = (uint32_t)gi * kStaticPerCta;
    const uint32_t cnt = a.n_envs - s0 < (uint32_t)kStaticPerCta ? a.n_envs - s0 : (uint32_t)kStaticPerCta;
    groups[gi] = Group{s0, (uint16_t)cnt, 0, 0u, s0};
  }
}

std::mutex g_mu;
uint8_t *g_addr[256] = {};

// Device address of g_scratch on the current device (looked up once per device).
int scratch_address(uint8_t **out) {
  int dev = 0;
  cudaError_t r = cudaGetDevice(&dev);
  if (r != cudaSuccess) return cuda_fail(r, "octax_rollout_static: cudaGetDevice");
  if (dev < 0 || dev >= 256) {
    set_error("octax_rollout_static: device ordinal out of range");
    return OCTAX_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    r = cudaGetSymbolAddress(&p, g_scratch);
    if (r != cudaSuccess) return cuda_fail(r, "octax_rollout_static: cudaGetSymbolAddress");
    g_addr[dev] = static_cast<uint8_t *>(p);
  }
  *out = g_addr[dev];
  return OCTAX_OK;
}

}  // namespace
}  // namespace octax

using namespace octax;

extern "C" int octax_rollout_static(const octax_game *game, int64_t n_envs, uint32_t quirks,
                                    uint64_t seed, int n_steps, const uint8_t *actions_dev,
                                    uint8_t *obs_dev, float *reward_dev, uint8_t *done_dev,
                                    void *cuda_stream) {
  if (!game || n_envs < 1 || n_steps < 1 || (quirks & ~0x3Fu)) {
    set_error("octax_rollout_static: need a game, n_envs >= 1, n_steps >= 1, known quirk bits");
    return OCTAX_EINVAL;
  }
  if (game->variant != OCTAX_VARIANT_CHIP8) {
    set_error("octax_rollout_static: CHIP-8 games only");
    return OCTAX_EINVAL;
  }
  if (n_envs > kStaticMaxEnvs) {
    set_error("octax_rollout_static: n_envs exceeds the static capacity of 1024 instances");
    return OCTAX_EINVAL;
  }
  if (!actions_dev || !obs_dev || !reward_dev || !done_dev ||
      (reinterpret_cast<uintptr_t>(obs_dev) & 15u)) {
    set_error("octax_rollout_static: actions, obs (16-byte aligned), reward and done are required");
    return OCTAX_EINVAL;
  }
  std::vector<GameDev> dev_games;
  std::vector<uint8_t> image;
  int rc = build_games(game, 1, dev_games, image);
  if (rc) return rc;
  uint8_t *base = nullptr;
  rc = scratch_address(&base);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

  DevState st{};
  size_t off = 0;
  void **dst[] = {(void **)&st.v,        (void **)&st.pcI,        (void **)&st.misc, (void **)&st.stack,
                  (void **)&st.disp,     (void **)&st.dirty,      (void **)&st.ram,  (void **)&st.ep,
                  (void **)&st.env_steps, (void **)&st.prev_score, (void **)&st.key,  (void **)&st.uid,
                  (void **)&st.out_row,  (void **)&st.game,   (void **)&st.last_act,
                  (void **)&st.mode,     (void **)&st.rpl,    (void **)&st.wrange};
  for (int i = 0; i < 18; ++i) {
    *dst[i] = base + off;
    off += up256(kArr[i]);
  }
  st.n = kStaticMaxEnvs;  // array stride; slots [0, n_envs) are used
  const GameDev *game_d = reinterpret_cast<const GameDev *>(base + kOffGame);
  const uint8_t *image_d = base + kOffImage;
  const Group *groups_d = reinterpret_cast<const Group *>(base + kOffGroups);
  const int n_groups = (int)((n_envs + kStaticPerCta - 1) / kStaticPerCta);

  for (int half = 0; half < 2; ++half) {
    SetupArgs a;
    memset(&a, 0, sizeof a);
    a.game = dev_games[0];
    memcpy(a.image_half, image.data() + half * (kRamBytes / 2), kRamBytes / 2);
    a.half = half;
    a.n_groups = n_groups;
    a.n_envs = (uint32_t)n_envs;
    static_setup_kernel<<<1, 256, 0, s>>>(a);
  }
  cudaError_t r = cudaGetLastError();
  if (r != cudaSuccess) return cuda_fail(r, "octax_rollout_static: setup launch");

  // reset every instance (this clears all state a step reads; RAM pages are
  // only read after this call writes them)
  ResetLaunch rp;
  memset(&rp, 0, sizeof rp);
  rp.st = st;
  rp.games = game_d;
  rp.images = image_d;
  rp.groups = groups_d;
  rp.n_groups = n_groups;
  rp.S = game->stack_frames;
  rp.quirks = quirks;
  rp.ipw = kStaticIpw;
  rp.init = 1;
  rp.seed = seed;
  rp.set_rows = 1;
  r = launch_reset(rp, kStaticBlock, s);
  if (r != cudaSuccess) return cuda_fail(r, "octax_rollout_static: reset launch");

  const int spl = 4;
  for (int s0 = 0; s0 < n_steps; s0 += spl) {
    StepLaunch p;
    memset(&p, 0, sizeof p);
    p.st = st;
    p.games = game_d;
    p.images = image_d;
    p.groups = groups_d;
    p.n_groups = n_groups;
    p.io0 = IO{actions_dev, obs_dev, reward_dev, done_dev, n_envs};
    p.step0 = s0;
    p.steps = n_steps - s0 < spl ? n_steps - s0 : spl;
    p.S = game->stack_frames;
    p.quirks = quirks;
    p.ipw = kStaticIpw;
    p.wrappers = uses_wrappers(dev_games.data(), 1);
    r = launch_step(p, n_groups, kStaticBlock, s);
    if (r != cudaSuccess) return cuda_fail(r, "octax_rollout_static: step launch");
  }
  return OCTAX_OK;
}
