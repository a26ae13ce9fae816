// The actor-critic network of §4.1 on the tensor cores (tcgen05, TMEM), and
// the rollout that runs it between environment steps on the device.
//
// Network (§4.1): the 4-frame stack in the (frame, x, y) = (4, 64, 32)
// orientation; conv1 32 filters (8,4)/(4,2) -> 15 x 15; conv2 64 filters 4/2
// -> 6 x 6; conv3 64 filters 3/1 -> 4 x 4; ReLU after each; flatten; actor
// and critic heads of 256 ReLU units; n_logits actor outputs and one value.
// VALID convolutions; weights and stored activations in bfloat16, products
// accumulated in fp32 (TMEM), heads' output layers in fp32 on the CUDA cores.
//
// Conv kernel (persistent, one CTA per SM: 8 warps that build operands and
// drain accumulators, and three threads in three more warps that issue the
// MMAs and bulk copies: an MMA costs its issuing thread more time than its
// share of the tensor pipe, so conv1's even pairs, its odd pairs and conv2's
// tiles come from different threads). A batch of kP = 8
// instances is processed at a time; the rows of every GEMM are
// (grid position, instance) with the instance fastest, so one 8-row core
// matrix of the tcgen05 no-swizzle K-major layout is one grid position of
// all 8 instances, and a position shift is a shift of the descriptor's start
// address by whole core matrices. Every convolution is then a sum over its
// kernel taps of GEMMs whose A operand is the layer input at a shifted start:
// no im2col copies.
//  - conv1 works on 4 x 2-pixel blocks: with stride (4, 2) its (8, 4) kernel
//    covers 2 x 2 blocks, so it is 4 taps of K = 32 (4 frames x 8 pixels)
//    over a 16 x 16 grid of blocks, expanded from the packed frame bits to
//    bf16 0/1; two output rows (16 positions x 8 instances = 128 rows each)
//    share one N = 64 accumulator fed by the three block rows they read.
//  - conv2 (stride 2) reads conv1's output split by the parity of x and y:
//    tap (kx, ky) reads sub-grid (kx & 1, ky & 1) at offset (kx >> 1,
//    ky >> 1) of an 8-wide grid. The taps kx and kx + 2 read the same
//    sub-grid one position apart, so they are stacked along N (N = 128) and
//    the drain adds columns 64..127 of row g + 1 to columns 0..63 of row g.
//    The sub-grids are kept as a band of four grid rows that slides down by
//    two with conv1's output rows; each M tile covers two output rows and
//    reads three grid rows, so the next conv1 pair writes the fourth while
//    the tile computes.
//  - conv3 (stride 1) reads conv2's output on an 8-wide grid. The three taps
//    kx of a kernel row ky read the same rows shifted by kx positions, so
//    they are stacked along N (N = 192: one MMA per ky and k-step reads its A
//    tile once for all three) and the shift is applied when draining: the
//    output at position g sums columns 0..63 of row g, 64..127 of row g + 1
//    and 128..191 of row g + 2.
//  Rows whose grid position lies outside the layer's output are computed
//  and discarded (they read padding or neighbouring positions, always inside
//  the buffers).
// Heads kernel: one CTA per (128-instance tile, head); K = 1024 streamed in
// 32-wide slices through a 3-stage ring (one thread issues the copies,
// another the MMAs); the actor CTA also draws the action.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "octax_internal.h"

struct octax_policy {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int n_logits = 0;
  int64_t max_envs = 0;
  int sms = 0;
  void *w1 = nullptr, *w2 = nullptr, *w3 = nullptr, *wh = nullptr;  // packed bf16
  float *fp = nullptr;        // biases and output layers (fp32), see FpLayout
  uint8_t *act3 = nullptr;    // flattened features, heads' A-operand tiles
  uint64_t *ring = nullptr;   // rollout: two packed observation slots [2][max_envs][4][32]
  unsigned int *err = nullptr;
  int stall = 0;              // octax_policy_debug_stall
};

namespace octax {

cudaStream_t env_stream(const octax_env *e);
int env_device(const octax_env *e);

namespace {

constexpr int kP = 8;            // instances per conv batch
constexpr int kThreads = 256;      // heads kernel: two warps per TMEM lane quarter
constexpr int kConvWork = 256;               // conv kernel: 8 warps build / drain (two per TMEM lane quarter)
constexpr int kConvThreads = kConvWork + 96; // + three warps whose first lanes issue the MMAs and bulk copies
constexpr int kIssuer = kConvWork;           // conv1's even pairs, conv3, the W1 / W2 copies and W3's first taps
constexpr int kIssuer2 = kConvWork + 32;     // conv2's tiles and the rest of W3
constexpr int kIssuer3 = kConvWork + 64;     // conv1's odd pairs
constexpr int kMaxLogits = 17;   // 16 keys + the no-op
constexpr uint64_t kMaxWaitNs = 1000000000ull;
constexpr uint32_t kMaxPolls = 1u << 24;

// ---- conv kernel shared memory (bytes) -------------------------------------
constexpr uint32_t kW1Off = 0;                             // conv1 B: [j 3][dx 2][chunk 4][n 64][8]
constexpr uint32_t kW1Bytes = 6 * 4 * 64 * 16;
constexpr uint32_t kW2Off = kW1Off + kW1Bytes;             // conv2 B: [ky 4][kx & 1][chunk 4][n 128][8]
constexpr uint32_t kW2Bytes = 4 * 2 * 4 * 128 * 16;
constexpr uint32_t kW3Bytes = 3 * 8 * 192 * 16;            // conv3 B: [ky 3][chunk 8][n = 64 kx + o][8]
constexpr uint32_t kSubPos = 33;                           // band: 4 grid rows of 8 + 1 pad position
constexpr uint32_t kSubBytes = kSubPos * 512;              // position: 4 chunks x 8 instances x 16 B
constexpr uint32_t kAct1Bytes = 4 * kSubBytes;             // 4 parity sub-grids
constexpr uint32_t kW3Off = kW2Off + kW2Bytes;             // W3 overlays frames + band (dead by then)
constexpr uint32_t kFrOff = kW3Off;                        // frames [32 rows][4][8] u64 during conv1
constexpr uint32_t kAct1Off = kW3Off + 8192;
constexpr uint32_t kW3RegionBytes = kW3Bytes > 8192 + kAct1Bytes ? kW3Bytes : 8192 + kAct1Bytes;
constexpr uint32_t kXOff = kW3Off + kW3RegionBytes;        // blocks (conv1) | conv2 output
constexpr uint32_t kBlkOff = kXOff;                        // 2 buffers x 49 block positions x 512 B
constexpr uint32_t kBlkBytes = 49 * 512;
constexpr uint32_t kAct2Off = kXOff;                       // 50 positions x (8 chunks x 8 x 16 B)
constexpr uint32_t kAct2Bytes = 50 * 1024;
constexpr uint32_t kXBytes = kAct2Bytes > 2 * kBlkBytes ? kAct2Bytes : 2 * kBlkBytes;
// conv2 / conv3 drain exchange: rows g + 1 and g + 2 of the warps that hold
// the last positions of a TMEM lane quarter come from the next quarter's
// warp: [supplier 2][channel half 2][lane 8 | 16][36 floats] (rows padded to
// 144 B: 16-byte aligned, and 8 lanes' rows start in distinct bank groups);
// conv2 tiles alternate between the two parts.
constexpr int kXbPitch = 36;
constexpr uint32_t kXbRow = kXbPitch * 4;
constexpr uint32_t kXb1Off = kXOff + kXBytes;              // part kx = 1: lanes 0..7
constexpr uint32_t kXb2Off = kXb1Off + 2 * 2 * 8 * kXbRow;  // part kx = 2: lanes 0..15
constexpr uint32_t kConvSmem = kXb2Off + 2 * 2 * 16 * kXbRow;
constexpr uint32_t kW3EarlyBytes = 8192;                   // W3 tap 0: loaded once the frames are dead
static_assert(kAct1Off + kAct1Bytes <= kXOff && kW3Off + kW3Bytes <= kXOff, "band and W3 inside their region");
static_assert(kFrOff + 8192 <= kAct1Off && kW3Off + kW3EarlyBytes <= kAct1Off, "frames / early W3 below the band");
static_assert(kConvSmem + 1024 <= 227 * 1024, "conv kernel shared memory (with 1 KB of static shared data)");

// TMEM columns (fp32) of the conv kernel's accumulators.
// conv1: 2 buffers x 2 output rows x 32; conv2: 3 tiles x 128; conv3: 2 tiles x 192
// (over conv1's and conv2's columns, all drained before conv3 is issued).
constexpr uint32_t kD1Col = 0, kD2Col = 128, kD3Col = 0, kConvTmemCols = 512;

// ---- heads kernel -----------------------------------------------------------
constexpr int kHeadStages = 3;
constexpr uint32_t kHA = 128 * 32 * 2;      // A slice: 128 rows x 32 K (bf16) = 4 chunk planes
constexpr uint32_t kHB = 256 * 32 * 2;      // B slice: 256 rows x 32 K
constexpr uint32_t kHeadOutOff = kHeadStages * (kHA + kHB);
constexpr uint32_t kHeadPartOff = kHeadOutOff + (kMaxLogits + 1) * 256 * 4 + 2 * 256 * 4;
constexpr uint32_t kHeadSmem = kHeadPartOff + 128 * (kMaxLogits + 1) * 4;  // + partial outputs of warps 4-7
constexpr uint32_t kAct3TileBytes = 128 * 1024 * 2;   // [slice 16][chunk 8][row 128][16 B]

// fp32 parameter block: b1 32 | b2 64 | b3 64 | bh [2][256] | wa2 [17][256] | ba2 [17] | wc2 [256] | bc2
struct FpLayout {
  static constexpr int b1 = 0, b2 = 32, b3 = 96, bh = 160, wa2 = 672, ba2 = wa2 + kMaxLogits * 256,
                       wc2 = ba2 + kMaxLogits, bc2 = wc2 + 256, total = bc2 + 1;
};

// ---- PTX helpers -------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0; i < kMaxPolls; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (global_ns() - t0 > kMaxWaitNs) break;
  }
  return false;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bulk copy global -> shared (16-byte aligned, size a multiple of 16), completing on `bar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, no swizzle: start, leading-dimension (K
// direction) and stride-dimension (M/N direction, between 8-row core
// matrices) byte offsets; bits 46-48 hold the fixed value 0b001.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}
// The descriptor of the same layout `bytes` further on: shared addresses stay
// below 2^18, so the 14-bit start field takes the offset without a carry, and
// the MMA-issuing loops add compile-time offsets to a base built once.
__device__ __forceinline__ uint64_t sdesc_at(uint64_t base, uint32_t bytes) { return base + (bytes >> 4); }
// Instruction descriptor, kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t M, uint32_t N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 32 consecutive fp32 columns of this thread's TMEM lane (warp w reads lanes 32w..32w+31).
__device__ __forceinline__ void tmem_ld32(uint32_t addr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(addr));
  // the wait names the loaded registers, so no use of them is scheduled before it
  asm volatile("tcgen05.wait::ld.sync.aligned;"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
        "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
        "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
        "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
      :
      : "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}
// Two 16-column loads (one per address) behind a single wait, in one asm
// statement so that no use of the registers can be scheduled before the wait.
__device__ __forceinline__ void tmem_ld16x2(uint32_t a0, uint32_t a1, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%33];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(a0), "r"(a1)
      : "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}
// 32 columns at each of a0, a1 (and a2) of this thread's TMEM lane, behind one wait.
__device__ __forceinline__ void tmem_ld32x2(uint32_t a0, uint32_t a1, float (&v)[32], float (&w)[32]) {
  uint32_t r[32], q[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(a0));
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]), "=r"(q[8]),
        "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]), "=r"(q[15]), "=r"(q[16]),
        "=r"(q[17]), "=r"(q[18]), "=r"(q[19]), "=r"(q[20]), "=r"(q[21]), "=r"(q[22]), "=r"(q[23]), "=r"(q[24]),
        "=r"(q[25]), "=r"(q[26]), "=r"(q[27]), "=r"(q[28]), "=r"(q[29]), "=r"(q[30]), "=r"(q[31])
      : "r"(a1));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
        "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
        "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
        "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
      :
      : "memory");
  asm volatile(""
      : "+r"(q[0]), "+r"(q[1]), "+r"(q[2]), "+r"(q[3]), "+r"(q[4]), "+r"(q[5]), "+r"(q[6]), "+r"(q[7]),
        "+r"(q[8]), "+r"(q[9]), "+r"(q[10]), "+r"(q[11]), "+r"(q[12]), "+r"(q[13]), "+r"(q[14]), "+r"(q[15]),
        "+r"(q[16]), "+r"(q[17]), "+r"(q[18]), "+r"(q[19]), "+r"(q[20]), "+r"(q[21]), "+r"(q[22]), "+r"(q[23]),
        "+r"(q[24]), "+r"(q[25]), "+r"(q[26]), "+r"(q[27]), "+r"(q[28]), "+r"(q[29]), "+r"(q[30]), "+r"(q[31])
      :
      : "memory");  // after the wait (volatile statements keep their order)
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    v[j] = __uint_as_float(r[j]);
    w[j] = __uint_as_float(q[j]);
  }
}
// 32 floats to / from one 16-byte aligned exchange row, as 8 vector accesses.
__device__ __forceinline__ void xrow_put(float *row, const float (&v)[32]) {
#pragma unroll
  for (int c = 0; c < 8; ++c)
    reinterpret_cast<float4 *>(row)[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
}
__device__ __forceinline__ void xrow_get(const float *row, float (&v)[32]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float4 f = reinterpret_cast<const float4 *>(row)[c];
    v[4 * c] = f.x;
    v[4 * c + 1] = f.y;
    v[4 * c + 2] = f.z;
    v[4 * c + 3] = f.w;
  }
}
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // .x = a (low half)
  return *reinterpret_cast<uint32_t *>(&h);
}
// bias + ReLU on 8 values, packed to one 16-byte chunk of 8 bf16.
// (bias: 16-byte aligned shared memory, read as two vectors)
__device__ __forceinline__ uint4 relu_chunk(const float *v, const float *bias) {
  const float4 b0 = reinterpret_cast<const float4 *>(bias)[0], b1 = reinterpret_cast<const float4 *>(bias)[1];
  const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
  float o[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) o[j] = fmaxf(v[j] + bb[j], 0.0f);
  return make_uint4(pack_bf16(o[0], o[1]), pack_bf16(o[2], o[3]), pack_bf16(o[4], o[5]), pack_bf16(o[6], o[7]));
}

__device__ __forceinline__ uint32_t philox_w0(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                              uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return c0;
}

struct ConvArgs {
  const uint64_t *obs_words;  // [n][4][32] packed frames (or null)
  const uint8_t *obs_u8;      // [n][4][32][64] uint8 frames (or null)
  int64_t n;
  const uint8_t *w1, *w2, *w3;  // packed bf16 B operands
  const float *fp;              // FpLayout
  uint8_t *act3;                // [tiles][16][8][128][16 B]
  unsigned int *err;
  int stall;                    // diagnostic: the first conv1 commit is skipped (its wait runs out)
};

// One 32-column conv1 tile or 64-column conv2/conv3 tile: issue `taps` x
// `kks` MMAs (M = 128) accumulating into TMEM column `col`.
struct TileSpec {
  uint32_t a_base, a_lbo, a_sbo;
  uint32_t b_base, b_lbo, b_sbo;
};

template <bool kU8>
__global__ void __launch_bounds__(kConvThreads, 1) policy_conv_kernel(const ConvArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  // MMA completion: conv1 x2, conv2, conv3 x2; bulk copies: W1 + W2, W3 x2; the final
  // drain on the error path (bars[8], [12], [13], one per issuing thread); conv1 blocks
  // built x2 (per block buffer), band rows written (worker arrivals)
  __shared__ __align__(8) uint64_t bars[14];
  __shared__ uint32_t tmem_s;
  __shared__ __align__(16) float sb[160];    // b1 | b2 | b3 (offsets used are multiples of 8)
  __shared__ uint2 nib[16];                  // 4 pixel bits -> 4 bf16 0 / 1 (element k = bit k)
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const uint32_t sbase = smem_u32(sm);
  const uint32_t bar_c1_0 = smem_u32(&bars[0]), bar_c1_1 = smem_u32(&bars[1]);
  const uint32_t bar_c2 = smem_u32(&bars[2]), bar_c3a = smem_u32(&bars[3]), bar_c3b = smem_u32(&bars[7]);
  const uint32_t bar_w = smem_u32(&bars[4]), bar_w3a = smem_u32(&bars[5]), bar_w3b = smem_u32(&bars[6]);
  const uint32_t bar_blk0 = smem_u32(&bars[9]), bar_blk1 = smem_u32(&bars[11]), bar_band = smem_u32(&bars[10]);

  for (int j = t; j < 160; j += kConvThreads) sb[j] = a.fp[j];
  if (t < 16)  // 1.0 in bf16 is 0x3F80
    nib[t] = make_uint2((t & 1) * 0x3F80u | ((t >> 1) & 1) * 0x3F800000u,
                        ((t >> 2) & 1) * 0x3F80u | ((t >> 3) & 1) * 0x3F800000u);
  if (t == 0) {
    for (int j = 0; j < 9; ++j) mbar_init(smem_u32(&bars[j]), 1);
    for (int j = 9; j < 12; ++j) mbar_init(smem_u32(&bars[j]), kConvWork);
    mbar_init(smem_u32(&bars[12]), 1);
    mbar_init(smem_u32(&bars[13]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_s)),
                 "r"(kConvTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_s;
  if (t == kIssuer) {
    mbar_expect_tx(bar_w, kW1Bytes + kW2Bytes);
    bulk_g2s(sbase + kW1Off, a.w1, kW1Bytes, bar_w);
    for (uint32_t o = 0; o < kW2Bytes; o += 16384) bulk_g2s(sbase + kW2Off + o, a.w2 + o, 16384, bar_w);
  }
  // every exit from the batch loop tests ok right after a block-wide
  // reduction of every thread's outcome, so all threads leave it together
  bool ok = !__syncthreads_or(!mbar_wait(bar_w, 0));
  uint32_t ph_c1_0 = 0, ph_c1_1 = 0, ph_c2 = 0, ph_c3a = 0, ph_c3b = 0, ph_w3 = 0;  // ph_w3: both W3 barriers
  uint32_t ph_blk0 = 0, ph_blk1 = 0, ph_band = 0;  // issuing threads: conv1 blocks built, band rows written
  uint32_t w3_pend = 0;  // issuing threads: W3 copies issued and not yet waited for (bit 0 early, bit 1 rest)
  const int64_t n_batches = (a.n + kP - 1) / kP;
  static_assert(kP * 64 == 2 * kConvWork, "two packed-frame pieces per worker");
  // a worker's two pieces of a batch's packed frames (q = t, t + 256:
  // instance q & 7, frame (q >> 7) & 3, rows 2 y2 and 2 y2 + 1, y2 = (q >> 3) & 15)
  auto load_frames = [&](int64_t first, uint4 &v0, uint4 &v1) {
    uint4 v[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int q = t + kConvWork * k, i = q & 7, c = (q >> 7) & 3, y2 = (q >> 3) & 15;
      if (first + i < a.n)
        v[k] = __ldg(reinterpret_cast<const uint4 *>(a.obs_words + (first + i) * 128 + c * 32 + 2 * y2));
    }
    v0 = v[0];
    v1 = v[1];
  };
  uint4 pf[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
  bool pf_ok = false;
  // warps w and w + 4 read the same TMEM lane quarter (rows 32 (w & 3) ..), each
  // one half of the accumulator's columns
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  const int half = warp >> 2;
  const bool issuer = warp >= kConvWork / 32;  // the MMA-issuing warps take no part in building / draining
  const int r = 32 * (warp & 3) + lane;  // M-tile row of this thread (TMEM lane)
  // base descriptors of every MMA operand (the issuing loops add constant offsets)
  const uint64_t a1d0 = sdesc(sbase + kBlkOff, 128, 512), a1d1 = sdesc(sbase + kBlkOff + kBlkBytes, 128, 512);
  const uint64_t b1d = sdesc(sbase + kW1Off, 1024, 128);
  const uint64_t a2d = sdesc(sbase + kAct1Off, 128, 512), b2d = sdesc(sbase + kW2Off, 2048, 128);
  const uint64_t a3d = sdesc(sbase + kAct2Off, 128, 1024), b3d = sdesc(sbase + kW3Off, 3072, 128);
  const int g = r >> 3, ri = r & 7;      // grid position in the tile, instance in the batch

  // wait for the next phase of a barrier (block-uniform outcome; also a block barrier)
  auto wait_all = [&](uint32_t bar, uint32_t &phase) -> bool {
    const bool w_ok = mbar_wait(bar, phase);
    phase ^= 1u;
    return !__syncthreads_or(!w_ok);
  };
  // the same among the 8 worker warps only (named barrier 1), so that they
  // need not wait for the issuing thread while it is issuing
  auto wait_workers = [&](uint32_t bar, uint32_t &phase) -> bool {
    const uint32_t w_ok = mbar_wait(bar, phase);
    phase ^= 1u;
    uint32_t any_fail;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.eq.u32 p, %1, 0;\n\tbarrier.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(any_fail)
        : "r"(w_ok), "r"(kConvWork)
        : "memory");
    return !any_fail;
  };

  for (int64_t batch = blockIdx.x; batch < n_batches && ok; batch += gridDim.x) {
    const int64_t i0 = batch * kP;
    // ---- frames of the batch, packed (bit x of row word y = pixel (x, y)),
    // stored [row y][frame c][instance i] so that the 32 lanes of a warp
    // building one block position read 32 consecutive words
    uint64_t *fr = reinterpret_cast<uint64_t *>(sm + kFrOff);
    if (!kU8) {
      // each worker's two 16-byte pieces (q = t, t + 256): loaded during the
      // previous batch's last drain (pf_ok), else here
      if (!issuer && !pf_ok) {
        load_frames(i0, pf[0], pf[1]);
      }
      pf_ok = false;
      for (int k = 0; k < 2 && !issuer; ++k) {  // instance i, frame c, rows 2 y2, 2 y2 + 1
        const int q = t + kConvWork * k, i = q & 7, c = (q >> 7) & 3, y2 = (q >> 3) & 15;
        fr[((2 * y2) * 4 + c) * 8 + i] = (uint64_t)pf[k].x | (uint64_t)pf[k].y << 32;
        fr[((2 * y2 + 1) * 4 + c) * 8 + i] = (uint64_t)pf[k].z | (uint64_t)pf[k].w << 32;
      }
    } else {
      for (int q = issuer ? kP * 128 : t; q < kP * 128; q += kConvWork) {  // one 64-byte row each
        const int i = q & 7, c = (q >> 8) & 3, y = (q >> 3) & 31;
        uint64_t bits = 0;
        if (i0 + i < a.n) {
          const uint4 *src = reinterpret_cast<const uint4 *>(a.obs_u8 + ((i0 + i) * 128 + c * 32 + y) * 64);
#pragma unroll
          for (int k4 = 0; k4 < 4; ++k4) {
            const uint4 v = __ldg(src + k4);
            const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
              for (int bb = 0; bb < 4; ++bb)
                bits |= (uint64_t)(((w4[k] >> (8 * bb)) & 0xFFu) != 0u) << (16 * k4 + 4 * k + bb);
          }
        }
        fr[(y * 4 + c) * 8 + i] = bits;
      }
    }
    __syncthreads();

    // ---- conv1 rows 0..13 (row 14 is never read by conv2) in 7 pairs,
    // software-pipelined: the blocks of pair p + 1 are built and its 16 MMAs
    // issued (second block buffer, second pair of TMEM accumulators) before
    // pair p's epilogue; conv2 runs on each completed band of three grid rows
    // while conv1 continues.
    // Blocks of block rows 2p .. 2p + 2 (position b = bx + 16 (by - 2p)); the
    // pad position 48 is read by discarded rows only. Warp w builds positions
    // 6w .. 6w + 5; lane = frame * 8 + instance; a 16-entry table turns 4
    // pixel bits into 4 bf16 elements.
    auto build = [&](int pr, int buf) {
      if (issuer) return;
      uint8_t *blk = sm + kBlkOff + buf * kBlkBytes;
      // a warp's 6 positions span at most two block rows: load their row words once
      const int r0 = (6 * warp) >> 4, r1 = (6 * warp + 5) >> 4;
      const int y0 = 2 * (2 * pr + r0), y1 = 2 * (2 * pr + r1);
      const uint64_t a0 = fr[y0 * 32 + lane], a1 = fr[(y0 + 1) * 32 + lane];
      const uint64_t b0 = fr[y1 * 32 + lane], b1 = fr[(y1 + 1) * 32 + lane];
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const int b = 6 * warp + j, bx = b & 15;
        const bool first = (b >> 4) == r0;
        const uint2 lo = nib[(uint32_t)((first ? a0 : b0) >> (4 * bx)) & 15u];
        const uint2 hi = nib[(uint32_t)((first ? a1 : b1) >> (4 * bx)) & 15u];
        *reinterpret_cast<uint4 *>(blk + b * 512 + lane * 16) = make_uint4(lo.x, lo.y, hi.x, hi.y);
      }
    };
    // Both output rows of the pair in one N = 64 accumulator: block row j
    // (shift dx) feeds row 2p through tap (dx, dy = j) and row 2p + 1 through
    // tap (dx, dy = j - 1); W1 holds, per (j, dx), those two taps stacked
    // over n (zeros where a tap does not apply), so each MMA reads its A tile
    // once for 64 outputs.
    auto issue_c1 = [&](int buf, bool first) {  // the issuing thread: output rows 2p, 2p + 1
      tc_fence_after();
      for (int j = 0; j < 3; ++j)
        for (int dx = 0; dx < 2; ++dx)
          for (int kk = 0; kk < 2; ++kk) {
            const uint64_t ad = sdesc_at(buf ? a1d1 : a1d0, (16 * j + dx) * 512 + kk * 256);
            const uint64_t bd = sdesc_at(b1d, (2 * j + dx) * 4096 + kk * 2048);
            mma_bf16(tmem + kD1Col + 64 * buf, ad, bd, idesc_bf16(128, 64), (j | dx | kk) != 0);
          }
      if (!(a.stall && first)) mma_commit(buf ? bar_c1_1 : bar_c1_0);
    };
    auto issue_c2 = [&](int tt) {  // the issuing thread: conv2 tile tt (output rows 2tt, 2tt + 1)
      tc_fence_after();
      for (int ky = 0; ky < 4; ++ky)
        for (int px = 0; px < 2; ++px) {  // taps (px, ky) and (px + 2, ky)
          const uint32_t sg = px + 2 * (ky & 1), shift = 8 * (ky >> 1);
          for (int kk = 0; kk < 2; ++kk) {
            const uint64_t ad = sdesc_at(a2d, sg * kSubBytes + shift * 512 + kk * 256);
            const uint64_t bd = sdesc_at(b2d, (ky * 2 + px) * 8192 + kk * 4096);
            mma_bf16(tmem + kD2Col + 128 * tt, ad, bd, idesc_bf16(128, 128), (ky | px | kk) != 0);
          }
        }
      mma_commit(bar_c2);
    };
    // The workers and the two issuing threads meet only through mbarriers
    // here. The workers arrive on blk[p & 1] when pair p's blocks are built,
    // which also says that pair p - 2 has been drained, so its TMEM buffer is
    // free (one barrier per block buffer: the next arrival on it needs pair
    // p's MMAs, issued only after the issuing thread of pairs p & 1 has
    // waited, so it never falls two phases behind a parity wait). They arrive on band
    // when the band rows of pairs 2, 4 and 6 are written; conv2's issuing
    // thread waits for it (the next arrival needs a conv1 pair whose MMAs come
    // after the tile's wait in the tensor pipe's order, through the slide's
    // wait for the tile). Each worker waits for the MMAs itself, so the
    // workers go on while an issuing thread sits in a full MMA queue. Every
    // wait is bounded; one that runs out only clears r_ok, and each side still
    // runs its whole schedule (no other side waits on it for long).
    bool r_ok = true;
    if (!issuer) {
      build(0, 0);
      fence_async_smem();
      mbar_arrive(bar_blk0);
      for (int pr = 0; pr < 7; ++pr) {
        const int cb = pr & 1, nb = cb ^ 1;
        if (pr + 1 < 7) {  // buffer nb: pair pr - 1's MMAs done (waited for last iteration)
          build(pr + 1, nb);
          fence_async_smem();
          mbar_arrive(nb ? bar_blk1 : bar_blk0);
        }
        r_ok &= mbar_wait(cb ? bar_c1_1 : bar_c1_0, cb ? ph_c1_1 : ph_c1_0);
        if (cb) ph_c1_1 ^= 1u; else ph_c1_0 ^= 1u;
        if (pr == 4 || pr == 6) {  // the previous tile must finish before its rows are rewritten
          r_ok &= mbar_wait(bar_c2, ph_c2);
          ph_c2 ^= 1u;
          asm volatile("bar.sync 1, %0;" ::"r"(kConvWork) : "memory");  // every worker's rows written
          // slide: grid rows 2, 3 -> 0, 1 (4 sub-grids x 16 positions x 512 B)
          for (int q = t; q < 4 * 16 * 32; q += kConvWork) {
            const int sgq = q >> 9, rem = q & 511;
            uint4 *base = reinterpret_cast<uint4 *>(sm + kAct1Off + sgq * kSubBytes);
            base[rem] = base[16 * 32 + rem];
          }
          asm volatile("bar.sync 1, %0;" ::"r"(kConvWork) : "memory");
        }
        tc_fence_after();
        {
          float v[32];  // columns 16 half .. of row 2p (v[0..15]) and of row 2p + 1 (v[16..31])
          const uint32_t d = tmem + lane_base + kD1Col + 64 * cb + 16 * half;
          tmem_ld16x2(d, d + 32, v);
          const int ox = g;
#pragma unroll
          for (int s2 = 0; s2 < 2; ++s2) {
            const int oy = 2 * pr + s2;
            if (ox <= 13) {  // conv2 reads x <= 13
              const int band = pr < 4 ? 0 : (pr < 6 ? 1 : 2);  // band b holds grid rows 2b .. 2b + 3
              const int slot = pr - 2 * band;                   // this pair's grid row is oy >> 1 = pr
              const int sg = (ox & 1) + 2 * (oy & 1);
              uint8_t *dst = sm + kAct1Off + sg * kSubBytes + ((ox >> 1) + 8 * slot) * 512 + ri * 16;
#pragma unroll
              for (int c = 0; c < 2; ++c)
                *reinterpret_cast<uint4 *>(dst + (2 * half + c) * 128) =
                    relu_chunk(v + 16 * s2 + 8 * c, sb + 16 * half + 8 * c);
            }
          }
        }
        tc_fence_before();
        if (pr == 2 || pr == 4 || pr == 6) {
          fence_async_smem();
          mbar_arrive(bar_band);
        }
      }
      // (the issuing warps skip the waits on conv2 tiles 0 and 1: two parity
      // flips, so their ph_c2 agrees with the workers' again here)
    } else if (t == kIssuer || t == kIssuer3) {  // conv1's even / odd pairs
      for (int pr = t == kIssuer ? 0 : 1; pr < 7; pr += 2) {
        const int b = pr & 1;
        r_ok &= mbar_wait(b ? bar_blk1 : bar_blk0, b ? ph_blk1 : ph_blk0);
        if (b) ph_blk1 ^= 1u; else ph_blk0 ^= 1u;
        issue_c1(pr & 1, pr == 0);
        if (pr == 6) {  // the frames are dead: W3 taps 0-1 into their place
          mbar_expect_tx(bar_w3a, kW3EarlyBytes);
          bulk_g2s(sbase + kW3Off, a.w3, kW3EarlyBytes, bar_w3a);
          w3_pend |= 1u;
        }
      }
    } else if (t == kIssuer2) {  // conv2 tiles as the band fills (rows of pairs 2, 4 and 6)
      for (int tt = 0; tt < 3; ++tt) {
        r_ok &= mbar_wait(bar_band, ph_band);
        ph_band ^= 1u;
        issue_c2(tt);
      }
    }
    // (no block barrier here: the drains of conv2 tiles 0 and 1 below need
    // only the workers' own waits, and conv2's issuing thread may still be
    // issuing tile 2; r_ok joins the block-wide wait on tile 2)
    // ---- conv2 epilogues into region X: tiles 0 and 1 (done) while tile 2
    // computes; conv2's issuing thread loads the rest of W3 over the band as soon
    // as tile 2 is done
    // Output g (valid for px = g & 7 < 6) adds row g + 1's second half: by a
    // shuffle, or for g = 3, 11 from the next lane quarter (rows 4, 12)
    // through the exchange buffer.
    auto drain_c2 = [&](int tt) {
      const int px = g & 7, py = 2 * tt + (g >> 3), h = half, qt = warp & 3;
      float *xb = reinterpret_cast<float *>(sm + ((tt & 1) ? kXb2Off : kXb1Off)) + ((qt >> 1) * 2 + h) * 8 * kXbPitch;
      float v[32], w[32];
      const uint32_t d = tmem + lane_base + kD2Col + 128 * tt + 32 * h;
      tmem_ld32x2(d, d + 64, v, w);
      if ((qt & 1) && lane < 8) xrow_put(xb + lane * kXbPitch, w);
#pragma unroll
      for (int c = 0; c < 32; ++c) w[c] = __shfl_down_sync(0xFFFFFFFFu, w[c], 8);
      asm volatile("bar.sync 1, %0;" ::"r"(kConvWork) : "memory");
      if (!(qt & 1) && lane >= 24) xrow_get(xb + (lane - 24) * kXbPitch, w);
#pragma unroll
      for (int c = 0; c < 32; ++c) v[c] += w[c];
      if (px < 6) {
        uint8_t *dst = sm + kAct2Off + (px + 8 * py) * 1024 + ri * 16;
#pragma unroll
        for (int c = 0; c < 4; ++c)
          *reinterpret_cast<uint4 *>(dst + (4 * h + c) * 128) = relu_chunk(v + 8 * c, sb + 32 + 32 * h + 8 * c);
      }
    };
    if (issuer) {
      if (t == kIssuer2 && mbar_wait(bar_c2, ph_c2)) {  // (a timeout here shows in the waits below)
        fence_async_smem();
        mbar_expect_tx(bar_w3b, kW3Bytes - kW3EarlyBytes);
        for (uint32_t o = kW3EarlyBytes; o < kW3Bytes; o += 16384)
          bulk_g2s(sbase + kW3Off + o, a.w3 + o, 16384, bar_w3b);
        w3_pend |= 2u;
      }
    } else {
      tc_fence_after();
      drain_c2(0);
      drain_c2(1);
    }
    {  // conv2 tile 2, and every thread's outcome so far
      const bool w_ok = mbar_wait(bar_c2, ph_c2) && ok && r_ok;
      ph_c2 ^= 1u;
      ok = !__syncthreads_or(!w_ok);
    }
    if (!ok) break;
    tc_fence_after();
    if (!issuer) drain_c2(2);
    tc_fence_before();
    fence_async_smem();
    ok = !__syncthreads_or(!(mbar_wait(bar_w3a, ph_w3) && mbar_wait(bar_w3b, ph_w3)));
    ph_w3 ^= 1u;
    w3_pend = 0;
    if (!ok) break;

    // ---- conv3: two tiles of 16 positions (qx + 8 qy, qy in {2u, 2u + 1}),
    // 3 kernel rows x 4 k-steps of N = 192 each (one completion barrier per
    // tile, so the first tile drains while the second computes)
    if (t == kIssuer) {
      tc_fence_after();
      for (int u = 0; u < 2; ++u) {
        for (int ky = 0; ky < 3; ++ky)
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t ad = sdesc_at(a3d, (16 * u + 8 * ky) * 1024 + kk * 256);
            const uint64_t bd = sdesc_at(b3d, ky * 24576 + kk * 6144);
            mma_bf16(tmem + kD3Col + 192 * u, ad, bd, idesc_bf16(128, 192), (ky | kk) != 0);
          }
        mma_commit(u ? bar_c3b : bar_c3a);
      }
    }
    // Drain: the outputs (qx < 4) lie in lane quarters 0 and 2 (positions
    // g = 0..3, 8..11); rows g + 1 and g + 2 come from the same warp by
    // shuffles, or, past the quarter's end, from quarters 1 and 3 (positions
    // 4, 5 and 12, 13, no outputs of their own) through the exchange buffer.
    // (the issuing warps go on to the batch's closing barrier; the workers'
    // outcome joins it there)
    for (int u = 0; u < 2 && !issuer; ++u) {
      ok = (u ? wait_workers(bar_c3b, ph_c3b) : wait_workers(bar_c3a, ph_c3a)) && ok;
      if (!ok) continue;  // uniform among the workers
      if (!kU8 && u == 1 && batch + gridDim.x < n_batches) {  // the next batch's frames, in flight during this drain
        load_frames((batch + gridDim.x) * kP, pf[0], pf[1]);
        pf_ok = true;
      }
      tc_fence_after();
      const int qt = warp & 3, h = half, sup = qt >> 1;
      const uint32_t d = tmem + lane_base + kD3Col + 192 * u + 32 * h;
      float *xb1 = reinterpret_cast<float *>(sm + kXb1Off) + (sup * 2 + h) * 8 * kXbPitch;
      float *xb2 = reinterpret_cast<float *>(sm + kXb2Off) + (sup * 2 + h) * 16 * kXbPitch;
      float v[32], w[32], x[32];
      if (qt & 1) {  // supplier: rows 4 qt + 0, 1 for the previous quarter
        tmem_ld32x2(d + 64, d + 128, v, w);
        if (lane < 8) xrow_put(xb1 + lane * kXbPitch, v);
        if (lane < 16) xrow_put(xb2 + lane * kXbPitch, w);
        asm volatile("bar.sync 1, %0;" ::"r"(kConvWork) : "memory");
        continue;
      }
      tmem_ld32x2(d + 64, d + 128, w, x);
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        w[c] = __shfl_down_sync(0xFFFFFFFFu, w[c], 8);
        x[c] = __shfl_down_sync(0xFFFFFFFFu, x[c], 16);
      }
      tmem_ld32(d, v);
      asm volatile("bar.sync 1, %0;" ::"r"(kConvWork) : "memory");
      if (lane >= 24) xrow_get(xb1 + (lane - 24) * kXbPitch, w);
      if (lane >= 16) xrow_get(xb2 + (lane - 16) * kXbPitch, x);
#pragma unroll
      for (int c = 0; c < 32; ++c) v[c] += w[c] + x[c];
      const int m = 16 * u + g, qx = m & 7, qy = m >> 3;
      const int64_t inst = i0 + ri;
      if (qx < 4 && inst < a.n) {
        const int q = qx + 4 * qy;  // feature slice: k = 64 q + channel
        uint8_t *dst = a.act3 + (inst >> 7) * (int64_t)kAct3TileBytes + q * 16384 + (inst & 127) * 16;
#pragma unroll
        for (int c = 0; c < 4; ++c)
          *reinterpret_cast<uint4 *>(dst + (4 * h + c) * 2048) = relu_chunk(v + 8 * c, sb + 96 + 32 * h + 8 * c);
      }
    }
    tc_fence_before();
    ok = !__syncthreads_or(!ok);  // region X and the W3 region are rewritten by the next batch
  }
  if (!ok && t == 0) atomicOr(a.err, 1u);
  if (!ok && (t == kIssuer || t == kIssuer2 || t == kIssuer3)) {  // let this thread's MMAs and copies land
    const uint32_t fin = smem_u32(&bars[t == kIssuer ? 8 : (t == kIssuer2 ? 12 : 13)]);
    mma_commit(fin);
    mbar_wait(fin, 0);
    if (t == kIssuer) mbar_wait(bar_w, 0);
    if (w3_pend & 1u) mbar_wait(bar_w3a, ph_w3);
    if (w3_pend & 2u) mbar_wait(bar_w3b, ph_w3);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kConvTmemCols));
}

struct HeadsArgs {
  const uint8_t *act3;
  int64_t n;
  const uint8_t *wh;     // [2][16 slices][8 chunks][256][16 B]
  const float *fp;       // FpLayout
  int L;
  float *logits;         // [n][L] or null
  float *value;          // [n] or null
  uint8_t *actions;      // [n] or null
  uint32_t key0, key1, step;
  unsigned int *err;
};

// blockIdx.x: 128-instance tile; blockIdx.y: 0 actor, 1 critic.
__global__ void __launch_bounds__(kThreads, 1) policy_heads_kernel(const HeadsArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t full[kHeadStages], empty[kHeadStages], fin;
  __shared__ uint32_t tmem_s;
  const int t = threadIdx.x, warp = t >> 5;
  const int head = blockIdx.y;
  const int64_t tile = blockIdx.x;
  const uint32_t sbase = smem_u32(sm);
  float *wout = reinterpret_cast<float *>(sm + kHeadOutOff);      // actor [L][256] or critic [256]
  float *bias = wout + (kMaxLogits + 1) * 256;                     // [256] hidden biases, then outputs'
  if (head == 0) {
    for (int j = t; j < a.L * 256; j += kThreads) wout[j] = a.fp[FpLayout::wa2 + j];
    for (int j = t; j < a.L; j += kThreads) bias[256 + j] = a.fp[FpLayout::ba2 + j];
  } else {
    for (int j = t; j < 256; j += kThreads) wout[j] = a.fp[FpLayout::wc2 + j];
    if (t == 0) bias[256] = a.fp[FpLayout::bc2];
  }
  for (int j = t; j < 256; j += kThreads) bias[j] = a.fp[FpLayout::bh + 256 * head + j];
  if (t == 0) {
    for (int s = 0; s < kHeadStages; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(&fin), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tmem_s)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_s;
  const uint8_t *A = a.act3 + tile * (int64_t)kAct3TileBytes;
  const uint8_t *B = a.wh + (int64_t)head * (16 * 8 * 256 * 16);
  constexpr int kSlices = 32;  // K = 1024 in slices of 32 (4 chunks)
  bool ok = true;
  // Thread 0 issues the copies, thread 32 the MMAs: each runs its own chain of
  // waits and issues (a bulk copy or an MMA costs far more latency on the
  // issuing thread than its bytes or its share of the tensor pipe).
  __shared__ int s_landed;  // slices whose copies the MMA thread has waited for
  int loaded = 0;           // thread 0: slices whose copies were issued
  if (t == 0) {
    for (int s = 0; s < kSlices && ok; ++s) {
      const int st = s % kHeadStages;
      // stage st last held slice s - kHeadStages: its MMAs must be done
      if (s >= kHeadStages) ok = mbar_wait(smem_u32(&empty[st]), ((s / kHeadStages) - 1) & 1);
      if (!ok) break;
      const uint32_t f = smem_u32(&full[st]);
      mbar_expect_tx(f, kHA + kHB);
      bulk_g2s(sbase + st * (kHA + kHB), A + (int64_t)s * kHA, kHA, f);
      bulk_g2s(sbase + st * (kHA + kHB) + kHA, B + (int64_t)s * kHB, kHB, f);
      loaded = s + 1;
    }
  } else if (t == 32) {
    int landed = 0;
    for (int s = 0; s < kSlices && ok; ++s) {
      const int st = s % kHeadStages;
      ok = mbar_wait(smem_u32(&full[st]), (s / kHeadStages) & 1);
      if (!ok) break;
      landed = s + 1;
      tc_fence_after();
      const uint32_t a0 = sbase + st * (kHA + kHB), b0 = a0 + kHA;
      for (int kk = 0; kk < 2; ++kk)
        mma_bf16(tmem, sdesc(a0 + kk * 2 * 2048, 2048, 128), sdesc(b0 + kk * 2 * 4096, 4096, 128),
                 idesc_bf16(128, 256), (s | kk) != 0);
      mma_commit(smem_u32(&empty[st]));
    }
    // the last slice's MMAs complete -> every earlier one has too
    if (ok) ok = mbar_wait(smem_u32(&empty[(kSlices - 1) % kHeadStages]), ((kSlices - 1) / kHeadStages) & 1);
    if (!ok) {  // let this thread's MMAs land before TMEM goes
      mma_commit(smem_u32(&fin));
      mbar_wait(smem_u32(&fin), 0);
    }
    s_landed = landed;
  }
  ok = !__syncthreads_or(!ok);
  if (!ok && t == 0)  // copies issued but never waited for land before shared memory goes
    for (int q = s_landed; q < loaded; ++q) mbar_wait(smem_u32(&full[q % kHeadStages]), (q / kHeadStages) & 1);
  tc_fence_after();
  // warps w and w + 4 read TMEM lane quarter w & 3 (instance t & 127), each
  // one half of the 256 hidden units; warps 4-7 hand their partial outputs
  // over through shared memory
  const int row = t & 127, hh = warp >> 2;
  const int64_t inst = tile * 128 + row;
  float *part = reinterpret_cast<float *>(sm + kHeadPartOff) + row * (kMaxLogits + 1);
  float acc[kMaxLogits];
#pragma unroll
  for (int j = 0; j < kMaxLogits; ++j) acc[j] = 0.0f;
  if (ok) {
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    // one output's dot product over 32 hidden units: the weights as 8 vector
    // loads, four independent partial sums
    auto dot32 = [&](const float(&h)[32], const float *w) -> float {
      const float4 *w4 = reinterpret_cast<const float4 *>(w);
      float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 ww = w4[q];
        s0 = fmaf(h[4 * q], ww.x, s0);
        s1 = fmaf(h[4 * q + 1], ww.y, s1);
        s2 = fmaf(h[4 * q + 2], ww.z, s2);
        s3 = fmaf(h[4 * q + 3], ww.w, s3);
      }
      return (s0 + s1) + (s2 + s3);
    };
    auto chunk = [&](float(&h)[32], int c0) {
#pragma unroll
      for (int j = 0; j < 32; ++j) h[j] = fmaxf(h[j] + bias[c0 + j], 0.0f);
      if (head == 0) {
#pragma unroll
        for (int o = 0; o < kMaxLogits; ++o)
          if (o < a.L) acc[o] += dot32(h, wout + o * 256 + c0);
      } else {
        acc[0] += dot32(h, wout + c0);
      }
    };
    for (int c0 = 128 * hh; c0 < 128 * hh + 128; c0 += 64) {  // two 32-column TMEM loads behind one wait
      float v[32], w[32];
      tmem_ld32x2(tmem + lane_base + c0, tmem + lane_base + c0 + 32, v, w);
      chunk(v, c0);
      chunk(w, c0 + 32);
    }
    if (hh) {
#pragma unroll
      for (int o = 0; o < kMaxLogits; ++o) part[o] = acc[o];
    }
  }
  __syncthreads();
  if (ok && !hh) {
#pragma unroll
    for (int o = 0; o < kMaxLogits; ++o) acc[o] += part[o];
    if (inst < a.n) {
      if (head == 0) {
        float m = -INFINITY;
#pragma unroll
        for (int o = 0; o < kMaxLogits; ++o)
          if (o < a.L) {
            acc[o] += bias[256 + o];
            m = fmaxf(m, acc[o]);
            if (a.logits) a.logits[inst * a.L + o] = acc[o];
          }
        if (a.actions) {
          // inverse CDF: the first index whose cumulative weight exceeds u * total
          const uint32_t w = philox_w0((uint32_t)inst, a.step, 0u, 0u, a.key0, a.key1);
          const float u = (float)(w >> 8) * 5.9604644775390625e-08f;  // 2^-24
          float e[kMaxLogits], tot = 0.0f;
#pragma unroll
          for (int o = 0; o < kMaxLogits; ++o) {
            e[o] = o < a.L ? expf(acc[o] - m) : 0.0f;
            tot += e[o];
          }
          const float target = u * tot;
          float run = 0.0f;
          int pick = a.L - 1;
          bool found = false;
#pragma unroll
          for (int o = 0; o < kMaxLogits; ++o) {
            run += e[o];
            if (o < a.L && !found && target < run) {
              pick = o;
              found = true;
            }
          }
          a.actions[inst] = (uint8_t)pick;
        }
      } else if (a.value) {
        a.value[inst] = acc[0] + bias[256];
      }
    }
  }
  if (!ok && t == 0) atomicOr(a.err, 1u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

// ---- host: weight packing ----------------------------------------------------
uint16_t bf16_bits(float f) {
  __nv_bfloat16 h = __float2bfloat16_rn(f);
  uint16_t b;
  std::memcpy(&b, &h, 2);
  return b;
}

int launch_forward(octax_policy *p, int64_t n, const uint64_t *obs_words, const uint8_t *obs_u8, uint64_t seed,
                   uint32_t step, float *logits, float *value, uint8_t *actions, cudaStream_t s) {
  if (n < 1 || n > p->max_envs) {
    set_error("octax_policy: need 1 <= n_envs <= max_envs of the policy");
    return OCTAX_EINVAL;
  }
  ConvArgs c{obs_words, obs_u8, n, (const uint8_t *)p->w1, (const uint8_t *)p->w2, (const uint8_t *)p->w3, p->fp,
             p->act3, p->err, p->stall};
  const int64_t batches = (n + kP - 1) / kP;
  const int grid = (int)std::min<int64_t>(batches, p->sms);
  if (obs_u8)
    policy_conv_kernel<true><<<grid, kConvThreads, kConvSmem, s>>>(c);
  else
    policy_conv_kernel<false><<<grid, kConvThreads, kConvSmem, s>>>(c);
  cudaError_t r = cudaGetLastError();
  if (r != cudaSuccess) return cuda_fail(r, "policy conv launch");
  HeadsArgs h{p->act3, n, (const uint8_t *)p->wh, p->fp, p->n_logits, logits, value, actions,
              (uint32_t)seed, (uint32_t)(seed >> 32), step, p->err};
  policy_heads_kernel<<<dim3((unsigned)((n + 127) / 128), 2), kThreads, kHeadSmem, s>>>(h);
  r = cudaGetLastError();
  if (r != cudaSuccess) return cuda_fail(r, "policy heads launch");
  return OCTAX_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace
}  // namespace octax

using namespace octax;

extern "C" {

int octax_policy_create(const octax_policy_params *prm, int64_t max_envs, int device, void *cuda_stream,
                        octax_policy **out) {
  if (!out || !prm || max_envs < 1 || max_envs > ((int64_t)1 << 31) || prm->n_logits < 1 ||
      prm->n_logits > kMaxLogits) {
    set_error("octax_policy_create: need params, out, 1 <= max_envs <= 2^31, 1 <= n_logits <= 17");
    return OCTAX_EINVAL;
  }
  *out = nullptr;
  const float *need[] = {prm->w1, prm->b1, prm->w2, prm->b2, prm->w3, prm->b3, prm->wa1,
                         prm->ba1, prm->wa2, prm->ba2, prm->wc1, prm->bc1, prm->wc2, prm->bc2};
  for (const float *q : need)
    if (!q) {
      set_error("octax_policy_create: every parameter array is required");
      return OCTAX_EINVAL;
    }
  cudaError_t r = cudaSetDevice(device);
  if (r != cudaSuccess) return cuda_fail(r, "octax_policy_create: cudaSetDevice");
  const int L = prm->n_logits;
  // conv1 B, per block row j (0..2) and shift dx: [j][dx][chunk = frame c][n 64][k' = kx + 4 ky];
  // n < 32: w1[n][c][4 dx + kx][2 j + ky] (tap dy = j, for j <= 1), n >= 32: w1[n - 32][c][4 dx + kx][2 (j - 1) + ky]
  // (tap dy = j - 1, for j >= 1), zero otherwise
  std::vector<uint16_t> w1p(6 * 4 * 64 * 8, 0);
  for (int j = 0; j < 3; ++j)
    for (int dx = 0; dx < 2; ++dx)
      for (int c = 0; c < 4; ++c)
        for (int n = 0; n < 64; ++n) {
          const int dy = n < 32 ? j : j - 1, o = n & 31;
          if (dy < 0 || dy > 1) continue;
          for (int k = 0; k < 8; ++k) {
            const int kx = 4 * dx + (k & 3), ky = 2 * dy + (k >> 2);
            w1p[(((j * 2 + dx) * 4 + c) * 64 + n) * 8 + k] = bf16_bits(prm->w1[((o * 4 + c) * 8 + kx) * 4 + ky]);
          }
        }
  // conv2 B: [ky][px = kx & 1][chunk j][n = 64 (kx >> 1) + o][e] = w2[o][8 j + e][kx][ky]
  // (taps kx and kx + 2 stacked along N)
  std::vector<uint16_t> w2p(4 * 2 * 4 * 128 * 8);
  for (int ky = 0; ky < 4; ++ky)
    for (int px = 0; px < 2; ++px)
      for (int j = 0; j < 4; ++j)
        for (int n = 0; n < 128; ++n)
          for (int e = 0; e < 8; ++e) {
            const int kx = px + 2 * (n >> 6), o = n & 63;
            w2p[((((ky * 2 + px) * 4 + j) * 128 + n) * 8) + e] =
                bf16_bits(prm->w2[((o * 32 + 8 * j + e) * 4 + kx) * 4 + ky]);
          }
  // conv3 B: [ky][chunk j][n = 64 kx + o][e] = w3[o][8 j + e][kx][ky] (the three taps of a
  // kernel row stacked along N)
  std::vector<uint16_t> w3p(3 * 8 * 192 * 8);
  for (int ky = 0; ky < 3; ++ky)
    for (int j = 0; j < 8; ++j)
      for (int n = 0; n < 192; ++n)
        for (int e = 0; e < 8; ++e) {
          const int kx = n >> 6, o = n & 63;
          w3p[((ky * 8 + j) * 192 + n) * 8 + e] = bf16_bits(prm->w3[((o * 64 + 8 * j + e) * 3 + kx) * 3 + ky]);
        }
  // heads B: [head][slice q (16)][chunk j][n 256][e]; feature k = 64 q + channel (q = qx + 4 qy),
  // the caller's flatten index is channel * 16 + qx * 4 + qy
  std::vector<uint16_t> whp(2 * 16 * 8 * 256 * 8);
  for (int head = 0; head < 2; ++head) {
    const float *W = head ? prm->wc1 : prm->wa1;
    for (int q = 0; q < 16; ++q)
      for (int j = 0; j < 8; ++j)
        for (int n = 0; n < 256; ++n)
          for (int e = 0; e < 8; ++e) {
            const int ch = 8 * j + e, qx = q & 3, qy = q >> 2;
            whp[((((size_t)head * 16 + q) * 8 + j) * 256 + n) * 8 + e] =
                bf16_bits(W[(size_t)n * 1024 + ch * 16 + qx * 4 + qy]);
          }
  }
  std::vector<float> fp(FpLayout::total, 0.0f);
  std::memcpy(&fp[FpLayout::b1], prm->b1, 32 * 4);
  std::memcpy(&fp[FpLayout::b2], prm->b2, 64 * 4);
  std::memcpy(&fp[FpLayout::b3], prm->b3, 64 * 4);
  std::memcpy(&fp[FpLayout::bh], prm->ba1, 256 * 4);
  std::memcpy(&fp[FpLayout::bh + 256], prm->bc1, 256 * 4);
  std::memcpy(&fp[FpLayout::wa2], prm->wa2, (size_t)L * 256 * 4);
  std::memcpy(&fp[FpLayout::ba2], prm->ba2, (size_t)L * 4);
  std::memcpy(&fp[FpLayout::wc2], prm->wc2, 256 * 4);
  fp[FpLayout::bc2] = prm->bc2[0];

  octax_policy *p = new octax_policy();
  p->device = device;
  p->n_logits = L;
  p->max_envs = max_envs;
  cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, device);
  if (p->sms < 1) p->sms = 1;
  const int64_t tiles = (max_envs + 127) / 128;
  auto fail = [&](cudaError_t e, const char *what) {
    octax_policy_destroy(p);
    return cuda_fail(e, what);
  };
  if ((r = cudaMalloc(&p->w1, w1p.size() * 2)) != cudaSuccess) return fail(r, "octax_policy_create: alloc");
  if ((r = cudaMalloc(&p->w2, w2p.size() * 2)) != cudaSuccess) return fail(r, "octax_policy_create: alloc");
  if ((r = cudaMalloc(&p->w3, w3p.size() * 2)) != cudaSuccess) return fail(r, "octax_policy_create: alloc");
  if ((r = cudaMalloc(&p->wh, whp.size() * 2)) != cudaSuccess) return fail(r, "octax_policy_create: alloc");
  if ((r = cudaMalloc((void **)&p->fp, fp.size() * 4)) != cudaSuccess) return fail(r, "octax_policy_create: alloc");
  if ((r = cudaMalloc((void **)&p->act3, (size_t)tiles * kAct3TileBytes)) != cudaSuccess)
    return fail(r, "octax_policy_create: alloc");
  if ((r = cudaMalloc((void **)&p->ring, (size_t)2 * max_envs * 1024)) != cudaSuccess)
    return fail(r, "octax_policy_create: alloc");
  if ((r = cudaMalloc((void **)&p->err, 4)) != cudaSuccess) return fail(r, "octax_policy_create: alloc");
  if (cuda_stream) {
    p->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if ((r = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking)) != cudaSuccess)
      return fail(r, "octax_policy_create: stream");
    p->own_stream = true;
  }
  r = cudaMemcpy(p->w1, w1p.data(), w1p.size() * 2, cudaMemcpyHostToDevice);
  if (r == cudaSuccess) r = cudaMemcpy(p->w2, w2p.data(), w2p.size() * 2, cudaMemcpyHostToDevice);
  if (r == cudaSuccess) r = cudaMemcpy(p->w3, w3p.data(), w3p.size() * 2, cudaMemcpyHostToDevice);
  if (r == cudaSuccess) r = cudaMemcpy(p->wh, whp.data(), whp.size() * 2, cudaMemcpyHostToDevice);
  if (r == cudaSuccess) r = cudaMemcpy(p->fp, fp.data(), fp.size() * 4, cudaMemcpyHostToDevice);
  if (r == cudaSuccess) r = cudaMemset(p->act3, 0, (size_t)tiles * kAct3TileBytes);
  if (r == cudaSuccess) r = cudaMemset(p->ring, 0, (size_t)2 * max_envs * 1024);
  if (r == cudaSuccess) r = cudaMemset(p->err, 0, 4);
  if (r == cudaSuccess)
    r = cudaFuncSetAttribute(policy_conv_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kConvSmem);
  if (r == cudaSuccess)
    r = cudaFuncSetAttribute(policy_conv_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kConvSmem);
  if (r == cudaSuccess)
    r = cudaFuncSetAttribute(policy_heads_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kHeadSmem);
  if (r != cudaSuccess) return fail(r, "octax_policy_create: upload");
  *out = p;
  return OCTAX_OK;
}

int octax_policy_forward(octax_policy *p, int64_t n_envs, const uint64_t *obs_words_dev, uint64_t seed, uint32_t step,
                         float *logits_dev, float *value_dev, uint8_t *actions_dev) {
  if (!p || !obs_words_dev || !aligned16(obs_words_dev)) {
    set_error("octax_policy_forward: need a policy and 16-byte aligned packed observations");
    return OCTAX_EINVAL;
  }
  cudaError_t r = cudaSetDevice(p->device);
  if (r != cudaSuccess) return cuda_fail(r, "octax_policy_forward: cudaSetDevice");
  return launch_forward(p, n_envs, obs_words_dev, nullptr, seed, step, logits_dev, value_dev, actions_dev,
                        p->stream);
}

int octax_policy_forward_u8(octax_policy *p, int64_t n_envs, const uint8_t *obs_dev, uint64_t seed, uint32_t step,
                            float *logits_dev, float *value_dev, uint8_t *actions_dev) {
  if (!p || !obs_dev || !aligned16(obs_dev)) {
    set_error("octax_policy_forward_u8: need a policy and 16-byte aligned observations");
    return OCTAX_EINVAL;
  }
  cudaError_t r = cudaSetDevice(p->device);
  if (r != cudaSuccess) return cuda_fail(r, "octax_policy_forward_u8: cudaSetDevice");
  return launch_forward(p, n_envs, nullptr, obs_dev, seed, step, logits_dev, value_dev, actions_dev, p->stream);
}

int octax_rollout_policy(octax_env *e, octax_policy *p, int n_steps, uint64_t seed, uint32_t step0,
                         uint64_t *obs_words_dev, uint8_t *actions_dev, float *logits_dev, float *value_dev,
                         float *reward_dev, uint8_t *done_dev) {
  if (!e || !p || n_steps < 1 || !obs_words_dev || !aligned16(obs_words_dev) || !actions_dev || !value_dev ||
      !reward_dev || !done_dev) {
    set_error("octax_rollout_policy: need env, policy, n_steps >= 1, aligned obs_words, actions, value, "
              "reward and done");
    return OCTAX_EINVAL;
  }
  const int64_t n = octax_num_envs(e);
  if (octax_stack_frames(e) != 4 || octax_variant(e) != OCTAX_VARIANT_CHIP8 || n > p->max_envs ||
      env_device(e) != p->device) {
    set_error("octax_rollout_policy: the network takes CHIP-8 environments with 4 stacked frames, at most "
              "max_envs instances, on the policy's device");
    return OCTAX_EINVAL;
  }
  cudaError_t r = cudaSetDevice(p->device);
  if (r != cudaSuccess) return cuda_fail(r, "octax_rollout_policy: cudaSetDevice");
  cudaStream_t s = env_stream(e);
  const size_t obs_bytes = (size_t)n * 1024;
  uint64_t *slot[2] = {p->ring, p->ring + (size_t)p->max_envs * 128};
  r = cudaMemcpyAsync(slot[0], obs_words_dev, obs_bytes, cudaMemcpyDeviceToDevice, s);
  if (r != cudaSuccess) return cuda_fail(r, "octax_rollout_policy: observation copy");
  int cur = 0;
  for (int k = 0; k < n_steps; ++k) {
    uint8_t *act = actions_dev + (size_t)k * n;
    int rc = launch_forward(p, n, slot[cur], nullptr, seed, step0 + (uint32_t)k,
                            logits_dev ? logits_dev + (size_t)k * n * p->n_logits : nullptr,
                            value_dev + (size_t)k * n, act, s);
    if (rc) return rc;
    rc = octax_step_n_packed(e, 1, act, slot[cur ^ 1], reward_dev + (size_t)k * n, done_dev + (size_t)k * n);
    if (rc) return rc;
    cur ^= 1;
  }
  r = cudaMemcpyAsync(obs_words_dev, slot[cur], obs_bytes, cudaMemcpyDeviceToDevice, s);
  if (r != cudaSuccess) return cuda_fail(r, "octax_rollout_policy: observation copy");
  return OCTAX_OK;
}

int octax_policy_sync(octax_policy *p) {
  if (!p) {
    set_error("octax_policy_sync: need a policy");
    return OCTAX_EINVAL;
  }
  cudaError_t r = cudaSetDevice(p->device);
  if (r == cudaSuccess) r = cudaStreamSynchronize(p->stream);
  if (r == cudaSuccess) r = cudaDeviceSynchronize();
  if (r != cudaSuccess) return cuda_fail(r, "octax_policy_sync");
  unsigned int h = 0;
  r = cudaMemcpy(&h, p->err, 4, cudaMemcpyDeviceToHost);
  if (r != cudaSuccess) return cuda_fail(r, "octax_policy_sync");
  if (h) {
    cudaMemset(p->err, 0, 4);
    set_error("octax_policy_sync: a policy kernel gave up a bounded wait; its outputs are incomplete");
    return OCTAX_ECUDA;
  }
  return OCTAX_OK;
}

int octax_policy_debug_stall(octax_policy *p, int on) {
  if (!p) {
    set_error("octax_policy_debug_stall: need a policy");
    return OCTAX_EINVAL;
  }
  p->stall = on != 0;
  return OCTAX_OK;
}

void octax_policy_destroy(octax_policy *p) {
  if (!p) return;
  cudaSetDevice(p->device);
  if (p->stream) cudaStreamSynchronize(p->stream);
  for (void *q : {p->w1, p->w2, p->w3, p->wh, (void *)p->fp, (void *)p->act3, (void *)p->ring, (void *)p->err})
    if (q) cudaFree(q);
  if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
  delete p;
}

}  // extern "C"
