// liboctax device code: the vectorised CHIP-8 environment step for sm_103a.
//
// Mapping (one CTA = one group of block/32 * ipw instances of one game):
//  - each warp emulates `ipw` instances, one per lane; PC/I/SP/timers/status,
//    the 64-bit dirty-page mask and the written-address range live in
//    registers; V0-VF (one u32 each),
//    the call stack and the bit-packed 64x32 display (one u64 per row, bit x =
//    pixel x; Super-CHIP: two u64 per row of the 128x64 buffer) live in
//    shared memory laid out [register|entry|row][instance],
//    so lanes touching their own instance never bank-conflict;
//  - the game's initial 4 KB RAM image (font + ROM) is staged once per CTA in
//    shared memory and is read-only; an instance's writes go to 64-byte pages
//    of its own RAM in global memory, tracked by the dirty mask. Fetches and
//    loads read the shared image unless the page is dirty; sprites read it
//    whenever their bytes lie outside the range of addresses written since
//    the reset (data packed next to a score buffer). A reset only clears the
//    mask and the range;
//  - observations can also be written one bit per pixel (the display words
//    themselves), 8x fewer bytes;
//  - dispatch limits divergence: the common opcodes (jumps, skips, loads,
//    adds, 8XYN ALU, key tests, FX07/FX15) run through one branch-free
//    predicated datapath that every lane executes together, with 8XYN as
//    integer multiply-adds from a per-N coefficient table; DXYN and four FX
//    forms take short branches, and the rest (CXNN, calls/returns, 00E0, BCD
//    and bulk memory ops, quirk variants, undefined encodings, the
//    Super-CHIP forms) a divergent switch. Every even address of the image
//    is decoded once per CTA into a micro-op (one bit per datapath decision,
//    NNN, and the pre-multiplied shared-memory offsets of VX and VY), so the
//    hot loop does one or two shared loads and single-bit tests per
//    instruction;
//  - observation frames are expanded from the packed rows by the whole warp
//    together (a byte of pixels becomes 8 bytes through a 256-entry table in
//    shared memory): every store is a 16-byte streaming store and each store
//    instruction writes eight complete 64-byte image rows (CHIP-8) or four
//    128-byte rows (Super-CHIP).
// Each instance runs exactly K instructions per frame, so all lanes of a warp
// meet at every frame boundary.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <cstring>

#include "octax_internal.h"

namespace octax {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// The CTA's dynamic shared memory. Every kernel lays it out with carve(), so
// the game's 4 KB RAM image is its first 4 KB. Reading the image through this
// array (not through a pointer) keeps those loads in the shared state space.
extern __shared__ __align__(16) uint8_t g_smem[];

__device__ __forceinline__ uint32_t img_byte(uint32_t a) { return g_smem[a]; }

struct Regs {
  uint32_t pc, I, sp, dt, st, status;
  uint64_t dirty;
  uint32_t draws, phase, env_steps;
  uint32_t key0, key1, uid;
  uint32_t last_act;  // action index applied at the previous step (sticky actions)
  uint32_t hires;     // SCHIP: 1 in 128x64 mode
  uint32_t wrange;    // lowest | highest << 16 RAM address written since the reset
};

struct Ctx {
  uint64_t *disp;      // shared: this instance's row 0; row r at disp[r * J]
  uint32_t *stack;     // shared: this instance's entry 0; entry i at stack[i * J]
  uint32_t *V;         // shared: this instance's V0; Vx at V[x * J]
  uint8_t *ram;        // global: this instance's 4 KB RAM (dirty pages)
  int J;
  const void *uops;      // shared: micro-op table, uint4 or uint2 entries (stage_game)
  const int4 *alu;       // shared: 8XYN coefficients, two int4 per N (stage_game)
  uint8_t *rpl;          // global: this instance's 16 SCHIP flag bytes
};

// Packed display words per instance and bytes per observation frame.
template <bool kS>
struct Disp {
  static constexpr int kWords = kS ? kSchipDispWords : kDispWords;
  static constexpr int kFrame = kS ? kSchipFrameBytes : kFrameBytes;
};

__device__ __forceinline__ uint32_t getV(const Ctx &C, uint32_t x) { return C.V[x * C.J]; }
__device__ __forceinline__ void setV(const Ctx &C, uint32_t x, uint32_t val) { C.V[x * C.J] = val & 0xFFu; }
__device__ __forceinline__ void setVF(const Ctx &C, uint32_t f) { C.V[15 * C.J] = f; }

__device__ __forceinline__ uint32_t dirty_bit(uint64_t dirty, uint32_t a) {
  return (uint32_t)(dirty >> ((a & 0xFFFu) >> kPageShift)) & 1u;
}

// Page copy-on-write keeps one 64-bit mask in registers, and beside it the
// range of RAM addresses written since the reset, so a sprite on a dirty
// page but outside that range (beside a score buffer, say) is still drawn
// from the shared image. Other reads of a dirty page use its complete copy.
// True when every byte of [a, a + len) (len <= 32, a + len <= 4096) is as in the image.
__device__ __forceinline__ bool unwritten(const Regs &R, const Ctx &C, uint32_t a, uint32_t len) {
  if (!(dirty_bit(R.dirty, a) | dirty_bit(R.dirty, a + len - 1u))) return true;
  return a + len - 1u < (R.wrange & 0xFFFFu) || a > (R.wrange >> 16);
}

// A byte of RAM: a dirty page's copy is complete.
__device__ __forceinline__ uint32_t rd8(const Regs &R, const Ctx &C, uint32_t a) {
  a &= 0xFFFu;
  return dirty_bit(R.dirty, a) ? (uint32_t)C.ram[a] : img_byte(a);
}

__device__ __forceinline__ void wr8(Regs &R, const Ctx &C, uint32_t a, uint32_t val) {
  a &= 0xFFFu;
  const uint32_t page = a >> kPageShift;
  if (!((R.dirty >> page) & 1u)) {  // first write to this page: copy it from the image
    const uint4 *src = reinterpret_cast<const uint4 *>(g_smem + (page << kPageShift));
    uint4 *dst = reinterpret_cast<uint4 *>(C.ram + (page << kPageShift));
    dst[0] = src[0];
    dst[1] = src[1];
    dst[2] = src[2];
    dst[3] = src[3];
    R.dirty |= 1ull << page;
  }
  R.wrange = min(R.wrange & 0xFFFFu, a) | max(R.wrange >> 16, a) << 16;
  C.ram[a] = (uint8_t)val;
}

// Philox4x32-10 (Salmon et al., SC'11); word 0 of the output block.
__device__ __forceinline__ uint32_t philox_w0(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1) {
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

__device__ __forceinline__ void tick(Regs &R) {
  R.dt -= (R.dt > 0);
  R.st -= (R.st > 0);
}

// DXYN: XOR an 8-wide, n-row sprite at (vx mod 64, vy mod 32); VF = collision.
__device__ __forceinline__ void draw(Regs &R, const Ctx &C, uint32_t vx, uint32_t vy, uint32_t n,
                                     uint32_t quirks) {
  const uint32_t x0 = vx & 63u, y0 = vy & 31u, I = R.I;
  const bool wrap = quirks & OCTAX_QUIRK_WRAP_SPRITES;
  // the sprite spans at most two pages: read it from the image unless a byte
  // of it may have been written
  const bool clean = n == 0 || (I + n <= (uint32_t)kRamBytes && unwritten(R, C, I, n));
  if (clean && !wrap && I + n <= (uint32_t)kRamBytes) {
    // Common case: sprite in the shared image, rows below the screen clipped,
    // no per-row checks; collision bits are OR-ed over the rows.
    const uint32_t rows = n < 32u - y0 ? n : 32u - y0;
    uint64_t *row = C.disp + y0 * C.J;
    uint64_t hit = 0;
    for (uint32_t r = 0; r < rows; ++r) {
      const uint64_t s = (uint64_t)(__brev(img_byte(I + r)) >> 24) << x0;  // pixel j -> bit x0 + j, right edge clips
      const uint64_t old = *row;
      hit |= old & s;
      *row = old ^ s;
      row += C.J;
    }
    setVF(C, hit != 0ull);
    return;
  }
  uint32_t coll = 0;
  for (uint32_t r = 0; r < n; ++r) {
    uint32_t py = y0 + r;
    if (py >= 32u) {
      if (!wrap) break;
      py &= 31u;
    }
    const uint32_t a = (I + r) & 0xFFFu;
    const uint32_t b = clean ? img_byte(a) : rd8(R, C, a);
    const uint32_t rev = __brev(b) >> 24;  // pixel j of the sprite -> bit j
    uint64_t s = (uint64_t)rev << x0;       // right edge clips
    if (wrap && x0 > 56u) s |= (uint64_t)rev >> (64u - x0);
    uint64_t *row = C.disp + py * C.J;
    const uint64_t old = *row;
    coll |= (old & s) != 0ull;
    *row = old ^ s;
  }
  setVF(C, coll);
}

// Each of the low 16 bits of v doubled (bit j -> bits 2j and 2j + 1).
__device__ __forceinline__ uint32_t double_bits(uint32_t v) {
  v = (v | (v << 8)) & 0x00FF00FFu;
  v = (v | (v << 4)) & 0x0F0F0F0Fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v | (v << 1);
}

// SCHIP DXYN / DXY0 on the 128x64 buffer (word 2y + h of an instance holds
// pixels 64h..64h+63 of row y, bit x = pixel 64h + x). In hires mode sprite
// pixels are buffer pixels; in lores mode the grid is 64x32 and each sprite
// pixel covers a 2x2 block. N = 0: 16x16 sprite, two bytes per row. VF = any
// lit buffer pixel turned off. Clipping (or the wrap quirk) on the grid.
__device__ __forceinline__ void draw_schip(Regs &R, const Ctx &C, uint32_t vx, uint32_t vy, uint32_t n,
                                           uint32_t quirks) {
  const bool wrap = quirks & OCTAX_QUIRK_WRAP_SPRITES;
  const uint32_t unit = R.hires ? 1u : 2u;               // buffer pixels per grid pixel
  const uint32_t gw = 128u / unit, gh = 64u / unit;      // grid
  const uint32_t x0 = vx & (gw - 1u), y0 = vy & (gh - 1u);
  const uint32_t rows = n ? n : 16u, width = n ? 8u : 16u;
  const uint32_t bx = x0 * unit, bits_w = width * unit;  // buffer column, pattern width (<= 32)
  // sprite bytes from the shared image unless one of them may have been written
  const uint32_t I = R.I, nbytes = n ? n : 32u;
  const bool from_img = I + nbytes <= (uint32_t)kRamBytes && unwritten(R, C, I, nbytes);
  uint32_t coll = 0;
  for (uint32_t r = 0; r < rows; ++r) {
    uint32_t gy = y0 + r;
    if (gy >= gh) {
      if (!wrap) break;
      gy -= gh;
    }
    uint32_t bits;
    if (from_img) bits = n ? img_byte(I + r) : (img_byte(I + 2u * r) << 8) | img_byte(I + 2u * r + 1u);
    else bits = n ? rd8(R, C, I + r) : ((rd8(R, C, I + 2u * r) << 8) | rd8(R, C, I + 2u * r + 1u));
    const uint32_t rev = __brev(bits) >> (32u - width);   // sprite pixel j -> bit j
    const uint64_t pat = unit == 1u ? (uint64_t)rev : (uint64_t)double_bits(rev);
    // pat << bx as a 128-bit value (lo, hi); bits past column 127 drop
    uint64_t lo = bx < 64u ? pat << bx : 0ull;
    uint64_t hi = bx == 0u ? 0ull : bx < 64u ? pat >> (64u - bx) : pat << (bx - 64u);
    if (wrap && bx + bits_w > 128u) lo |= pat >> (128u - bx);  // wrapped part re-enters at column 0
    for (uint32_t d = 0; d < unit; ++d) {
      uint64_t *row = C.disp + 2u * (gy * unit + d) * C.J;
      const uint64_t o0 = row[0], o1 = row[C.J];
      coll |= ((o0 & lo) | (o1 & hi)) != 0ull;
      row[0] = o0 ^ lo;
      row[C.J] = o1 ^ hi;
    }
  }
  setVF(C, coll);
}

// SCHIP scrolls of the 128x64 buffer by buffer pixels; vacated pixels clear.
__device__ __forceinline__ void scroll_down(const Ctx &C, uint32_t k) {
  for (int y = 63; y >= 0; --y)
    for (int h = 0; h < 2; ++h)
      C.disp[(2 * y + h) * C.J] = (uint32_t)y >= k ? C.disp[(2 * (y - (int)k) + h) * C.J] : 0ull;
}
__device__ __forceinline__ void scroll_right(const Ctx &C, uint32_t c) {  // 0 < c < 64
  for (int y = 0; y < 64; ++y) {
    const uint64_t lo = C.disp[2 * y * C.J], hi = C.disp[(2 * y + 1) * C.J];
    C.disp[2 * y * C.J] = lo << c;
    C.disp[(2 * y + 1) * C.J] = (hi << c) | (lo >> (64u - c));
  }
}
__device__ __forceinline__ void scroll_left(const Ctx &C, uint32_t c) {  // 0 < c < 64
  for (int y = 0; y < 64; ++y) {
    const uint64_t lo = C.disp[2 * y * C.J], hi = C.disp[(2 * y + 1) * C.J];
    C.disp[2 * y * C.J] = (lo >> c) | (hi << (64u - c));
    C.disp[(2 * y + 1) * C.J] = hi >> c;
  }
}

// Opcodes the predicated datapath covers: classes 1 3 4 6 7 A always; 5 9
// with N = 0; 8 with N in 0-7,E (classic shifts and logic); E with 9E/A1;
// F with 07 and 15. The rarer FX forms (0A 18 1E 29 ...) take the slow path,
// which keeps their selects out of every instruction slot.
__device__ __forceinline__ bool is_fast_op(uint32_t op, uint32_t quirks) {
  const uint32_t cls = op >> 12, n = op & 15u, nn = op & 0xFFu;
  const uint32_t cbit = 1u << cls;
  bool fast = (cbit & 0x04DAu) != 0;
  fast |= ((cbit & 0x0220u) != 0) & (n == 0);
  fast |= (cls == 8) & ((n <= 7) | (n == 14)) &
          ((quirks & (OCTAX_QUIRK_SHIFT_USES_VY | OCTAX_QUIRK_LOGIC_RESETS_VF)) == 0);
  fast |= (cls == 14) & ((nn == 0x9Eu) | (nn == 0xA1u));
  fast |= (cls == 15) & ((nn == 0x07u) | (nn == 0x15u));
  return fast;
}

// Decoded form of the opcode at an even image address, built once per CTA
// (the operands travel beside it: see fetch_uop). A slow opcode is stored raw
// (bit 20 clear). A fast one has one bit per datapath decision, so that each
// select tests a single bit:
//   bits 0-11 NNN (NN, N in its low bits) | 19 write VF (8XYN, N >= 4) | 20 fast |
//   21 skip negated | 22 skip | 23 skip compares VY (else NN) | 24 jump |
//   25 skip tests the held key | 26 VX = NN | 27 VX += NN | 28 VX = 8XYN |
//   29 VX = DT | 30 I = NNN | 31 DT = VX.
constexpr uint32_t kUopFast = 1u << 20;
// A slow opcode tagged for the short FX branch of execute (FX0A, FX18, FX29 and
// FX1E without its quirk): bit 21 set on the raw opcode (bit 20 clear).
constexpr uint32_t kUopFx = 1u << 21;

__device__ __forceinline__ uint32_t make_uop(uint32_t op, uint32_t quirks) {
  if (!is_fast_op(op, quirks)) {
    const uint32_t nn = op & 0xFFu;
    const bool fx = (op >> 12) == 0xFu &&
                    (nn == 0x0Au || nn == 0x18u || nn == 0x29u || (nn == 0x1Eu && !(quirks & OCTAX_QUIRK_FX1E_VF)));
    return fx ? (op | kUopFx) : op;
  }
  const uint32_t cls = op >> 12, nn = op & 0xFFu;
  uint32_t u = (op & 0xFFFu) | kUopFast;
  switch (cls) {
    case 0x1: u |= 1u << 24; break;
    case 0x3: u |= 1u << 22; break;
    case 0x4: u |= (1u << 22) | (1u << 21); break;
    case 0x5: u |= (1u << 22) | (1u << 23); break;
    case 0x9: u |= (1u << 22) | (1u << 23) | (1u << 21); break;
    case 0x6: u |= 1u << 26; break;
    case 0x7: u |= 1u << 27; break;
    case 0x8: u |= (1u << 28) | ((op & 15u) >= 4u ? (1u << 19) : 0u); break;
    case 0xA: u |= 1u << 30; break;
    case 0xE: u |= (1u << 22) | (1u << 25) | (nn == 0xA1u ? (1u << 21) : 0u); break;
    default:  // 0xF
      if (nn == 0x07u) u |= 1u << 29;
      else u |= 1u << 31;  // 0x15
      break;
  }
  return u;
}

// The rare / heavy instructions and every variant the fast datapath leaves
// out (quirk bits, undefined encodings). PC has already been advanced.
// kS: the SCHIP variant (128x64 buffer, extra 00xx and FXxx forms).
template <bool kS>
__device__ __forceinline__ void exec_slow(Regs &R, const Ctx &C, uint32_t op, uint32_t pc, int key,
                                       uint32_t quirks) {
  const uint32_t x = (op >> 8) & 15u, y = (op >> 4) & 15u, n = op & 15u, nn = op & 0xFFu;
  const uint32_t nnn = op & 0xFFFu;
  const uint32_t vx = getV(C, x), vy = getV(C, y);
  switch (op >> 12) {
    case 0x0:
      if (op == 0x00E0u) {
#pragma unroll 8
        for (int r = 0; r < Disp<kS>::kWords; ++r) C.disp[r * C.J] = 0ull;
      } else if (kS && (op & 0xFFF0u) == 0x00C0u) {  // scroll down N
        scroll_down(C, n * (R.hires ? 1u : 2u));
      } else if (kS && op == 0x00FBu) {  // scroll right 4
        scroll_right(C, R.hires ? 4u : 8u);
      } else if (kS && op == 0x00FCu) {  // scroll left 4
        scroll_left(C, R.hires ? 4u : 8u);
      } else if (kS && op == 0x00FDu) {  // exit: stay here
        R.status |= OCTAX_STATUS_EXIT;
        R.pc = pc;
      } else if (kS && (op == 0x00FEu || op == 0x00FFu)) {  // lores / hires, buffer kept
        R.hires = op & 1u;
      } else if (op == 0x00EEu) {
        if (R.sp == 0) {
          R.status |= OCTAX_STATUS_STACK_FAULT;
          R.sp = 16;
        }
        R.sp -= 1;
        R.pc = C.stack[R.sp * C.J];
      }
      break;
    case 0x1:
      R.pc = nnn;
      break;
    case 0x2:
      if (R.sp == 16) {
        R.status |= OCTAX_STATUS_STACK_FAULT;
        R.sp = 0;
      }
      C.stack[R.sp * C.J] = R.pc;
      R.sp += 1;
      R.pc = nnn;
      break;
    case 0x3:
      if (vx == nn) R.pc = (R.pc + 2u) & 0xFFFu;
      break;
    case 0x4:
      if (vx != nn) R.pc = (R.pc + 2u) & 0xFFFu;
      break;
    case 0x5:
      if (n) R.status |= OCTAX_STATUS_BAD_OP;
      else if (vx == vy) R.pc = (R.pc + 2u) & 0xFFFu;
      break;
    case 0x6:
      setV(C, x, nn);
      break;
    case 0x7:
      setV(C, x, vx + nn);
      break;
    case 0x8:
      switch (n) {
        case 0x0: setV(C, x, vy); break;
        case 0x1:
          setV(C, x, vx | vy);
          if (quirks & OCTAX_QUIRK_LOGIC_RESETS_VF) setVF(C, 0);
          break;
        case 0x2:
          setV(C, x, vx & vy);
          if (quirks & OCTAX_QUIRK_LOGIC_RESETS_VF) setVF(C, 0);
          break;
        case 0x3:
          setV(C, x, vx ^ vy);
          if (quirks & OCTAX_QUIRK_LOGIC_RESETS_VF) setVF(C, 0);
          break;
        case 0x4: {
          const uint32_t s = vx + vy;
          setV(C, x, s);
          setVF(C, s >> 8);
          break;
        }
        case 0x5:
          setV(C, x, vx - vy);
          setVF(C, vx >= vy);
          break;
        case 0x6: {
          const uint32_t src = (quirks & OCTAX_QUIRK_SHIFT_USES_VY) ? vy : vx;
          setV(C, x, src >> 1);
          setVF(C, src & 1u);
          break;
        }
        case 0x7:
          setV(C, x, vy - vx);
          setVF(C, vy >= vx);
          break;
        case 0xE: {
          const uint32_t src = (quirks & OCTAX_QUIRK_SHIFT_USES_VY) ? vy : vx;
          setV(C, x, src << 1);
          setVF(C, src >> 7);
          break;
        }
        default:
          R.status |= OCTAX_STATUS_BAD_OP;
          break;
      }
      break;
    case 0x9:
      if (n) R.status |= OCTAX_STATUS_BAD_OP;
      else if (vx != vy) R.pc = (R.pc + 2u) & 0xFFFu;
      break;
    case 0xA:
      R.I = nnn;
      break;
    case 0xB:
      R.pc = (nnn + ((quirks & OCTAX_QUIRK_JUMP_VX) ? vx : getV(C, 0))) & 0xFFFu;
      break;
    case 0xC: {
      const uint32_t rnd = philox_w0(R.uid, R.env_steps, pc | ((R.draws & 0xFFFFu) << 16), R.phase,
                                     R.key0, R.key1);
      R.draws += 1;
      setV(C, x, rnd & nn);
      break;
    }
    case 0xD:
      if (kS) draw_schip(R, C, vx, vy, n, quirks);
      else draw(R, C, vx, vy, n, quirks);
      break;
    case 0xE: {
      const bool pressed = key >= 0 && (uint32_t)key == (vx & 15u);
      if (nn == 0x9Eu) {
        if (pressed) R.pc = (R.pc + 2u) & 0xFFFu;
      } else if (nn == 0xA1u) {
        if (!pressed) R.pc = (R.pc + 2u) & 0xFFFu;
      } else {
        R.status |= OCTAX_STATUS_BAD_OP;
      }
      break;
    }
    default:  // 0xF
      switch (nn) {
        case 0x07: setV(C, x, R.dt); break;
        case 0x0A:
          if (key >= 0) setV(C, x, (uint32_t)key);
          else R.pc = pc;
          break;
        case 0x15: R.dt = vx; break;
        case 0x18: R.st = vx; break;
        case 0x1E: {
          const uint32_t s = R.I + vx;
          R.I = s & 0xFFFFu;
          if (quirks & OCTAX_QUIRK_FX1E_VF) setVF(C, s > 0xFFFu);
          break;
        }
        case 0x29: R.I = 0x50u + 5u * (vx & 15u); break;
        case 0x30:
          if (kS) R.I = kBigFontAddr + 10u * (vx & 15u);
          else R.status |= OCTAX_STATUS_BAD_OP;
          break;
        case 0x75:
          if (kS) {
            for (uint32_t i = 0; i <= x; ++i) C.rpl[i] = (uint8_t)getV(C, i);
          } else {
            R.status |= OCTAX_STATUS_BAD_OP;
          }
          break;
        case 0x85:
          if (kS) {
            for (uint32_t i = 0; i <= x; ++i) setV(C, i, C.rpl[i]);
          } else {
            R.status |= OCTAX_STATUS_BAD_OP;
          }
          break;
        case 0x33:
          wr8(R, C, R.I, vx / 100u);
          wr8(R, C, R.I + 1u, (vx / 10u) % 10u);
          wr8(R, C, R.I + 2u, vx % 10u);
          break;
        case 0x55:
          for (uint32_t i = 0; i <= x; ++i) wr8(R, C, R.I + i, getV(C, i));
          if (quirks & OCTAX_QUIRK_LOADSTORE_INC_I) R.I = (R.I + x + 1u) & 0xFFFFu;
          break;
        case 0x65:
          for (uint32_t i = 0; i <= x; ++i) setV(C, i, rd8(R, C, R.I + i));
          if (quirks & OCTAX_QUIRK_LOADSTORE_INC_I) R.I = (R.I + x + 1u) & 0xFFFFu;
          break;
        default:
          R.status |= OCTAX_STATUS_BAD_OP;
          break;
      }
      break;
  }
}

// Micro-op of the instruction at pc as {make_uop word, X * J, Y * J, NNN}:
// the shared-memory offsets of VX and VY come pre-multiplied. kW: the table
// holds those four words (one 16-byte load); otherwise it holds {word,
// X * J | Y * J << 16} (half the shared memory, two more extracts). Odd PCs
// and written pages give the raw opcode, which takes the general path.
template <bool kW>
__device__ __forceinline__ uint4 fetch_uop(const Regs &R, const Ctx &C, uint32_t pc) {
  if (!((pc & 1u) | dirty_bit(R.dirty, pc))) {
    if (kW) return static_cast<const uint4 *>(C.uops)[pc >> 1];
    const uint2 e = static_cast<const uint2 *>(C.uops)[pc >> 1];
    return make_uint4(e.x, e.y & 0xFFFFu, e.y >> 16, e.x & 0xFFFu);
  }
  return make_uint4((rd8(R, C, pc) << 8) | rd8(R, C, pc + 1u), 0u, 0u, 0u);
}

// Execute micro-op u, the instruction at R.pc. key: held CHIP-8 key or -1.
template <bool kS>
__device__ __forceinline__ void execute(Regs &R, const Ctx &C, const uint4 u4, int key, uint32_t quirks) {
  const uint32_t pc = R.pc, u = u4.x;
  if (u & kUopFast) {
    const uint32_t nnn = u4.w, nn = u & 0xFFu, n = u & 15u;
    uint32_t *const Vx = C.V + u4.y;
    const uint32_t vx = *Vx, vy = C.V[u4.z];
    // next PC: skips (bit 22; 23: against VY, 25: against the held key; 21: negated), jump (24)
    const uint32_t lhs = (u & (1u << 25)) ? (vx & 15u) : vx;
    const uint32_t rhs = (u & (1u << 25)) ? (uint32_t)key : ((u & (1u << 23)) ? vy : nn);
    const bool skip = (u & (1u << 22)) && ((lhs == rhs) != ((u & (1u << 21)) != 0u));
    uint32_t npc = (pc + (skip ? 4u : 2u)) & 0xFFFu;
    npc = (u & (1u << 24)) ? nnn : npc;
    R.pc = npc;
    // 8XYN result and flag (N in 0-7, E) as integer linear combinations, so
    // the work runs as multiply-adds (stage_game lists the coefficients):
    // result = c0 vx + c1 vy + c2 (vx & vy) + c3 (vx >> 1), whose low byte is
    // VX; the carry / NOT-borrow / shifted-out bit is bit 8 of a result + b vx + k.
    const int4 cr = C.alu[2 * n], cf = C.alu[2 * n + 1];
    const int32_t ix = (int32_t)vx, iy = (int32_t)vy;
    const int32_t res = cr.x * ix + cr.y * iy + cr.z * (ix & iy) + cr.w * (ix >> 1);
    const uint32_t alu = (uint32_t)res;
    const uint32_t flag = ((uint32_t)(cf.x * res + cf.y * ix + cf.z) >> 8) & 1u;
    // VX write (26: NN, 27: VX + NN, 28: 8XYN, 29: DT), VF (19), I = NNN (30), DT = VX (31)
    uint32_t val = (u & (1u << 27)) ? (vx + nn) : nn;
    val = (u & (1u << 28)) ? alu : val;
    val = (u & (1u << 29)) ? R.dt : val;
    if (u & (15u << 26)) *Vx = val & 0xFFu;
    if (u & (1u << 19)) C.V[15 * C.J] = flag;  // after VX: with X = F the flag wins
    R.I = (u & (1u << 30)) ? nnn : R.I;
    R.dt = (u & (1u << 31)) ? vx : R.dt;
  } else if (u & kUopFx) {  // FX0A / FX18 / FX1E / FX29: a short branch, not the general switch
    R.pc = (pc + 2u) & 0xFFFu;
    uint32_t *const Vx = C.V + u4.y;
    const uint32_t vx = *Vx, nn = u & 0xFFu;
    if (nn == 0x0Au) {
      if (key >= 0) *Vx = (uint32_t)key;
      else R.pc = pc;
    } else if (nn == 0x18u) {
      R.st = vx;
    } else if (nn == 0x1Eu) {
      R.I = (R.I + vx) & 0xFFFFu;
    } else {
      R.I = 0x50u + 5u * (vx & 15u);
    }
  } else if ((u >> 12) == 0xDu) {  // DXYN, the most frequent slow opcode: its own branch
    R.pc = (pc + 2u) & 0xFFFu;
    if (kS) draw_schip(R, C, getV(C, (u >> 8) & 15u), getV(C, (u >> 4) & 15u), u & 15u, quirks);
    else draw(R, C, getV(C, (u >> 8) & 15u), getV(C, (u >> 4) & 15u), u & 15u, quirks);
  } else {
    R.pc = (pc + 2u) & 0xFFFu;
    exec_slow<kS>(R, C, u & 0xFFFFu, pc, key, quirks);
  }
}

// Run `count` instructions.
template <bool kS, bool kW>
__device__ __forceinline__ void run_instrs(Regs &R, const Ctx &C, int key, uint32_t quirks,
                                           uint32_t count) {
  // Not unrolled: on divergent programs a second copy of the datapath costs
  // more in instruction fetch than the loop overhead it saves.
  for (uint32_t k = 0; k < count; ++k) execute<kS>(R, C, fetch_uop<kW>(R, C, R.pc), key, quirks);
}

__device__ __forceinline__ int32_t term_value(const Regs &R, const Ctx &C, const TermDev &t) {
  const int32_t v = t.src == OCTAX_SRC_REG ? (int32_t)getV(C, t.idx & 15u) : (int32_t)rd8(R, C, t.idx);
  switch (t.xform) {
    case OCTAX_X_RAW: return v;
    case OCTAX_X_NEG: return -v;
    case OCTAX_X_DEC_TENS: return v / 10;
    case OCTAX_X_DEC_ONES: return v % 10;
    case OCTAX_X_DEC_TENS_MINUS_ONES: return v / 10 - v % 10;
    case OCTAX_X_NIB_HI_MINUS_LO: return (v >> 4) - (v & 15);
    case OCTAX_X_ZERO_IF_GT: return v > t.arg ? 0 : v;
    default: return 0;
  }
}

__device__ __forceinline__ int32_t score(const Regs &R, const Ctx &C, const GameDev &G) {
  int32_t s = 0;
  for (uint32_t i = 0; i < G.n_score; ++i) s += term_value(R, C, G.score[i]);
  return s;
}

__device__ __forceinline__ bool terminated(const Regs &R, const Ctx &C, const GameDev &G) {
  bool hit = false;
  for (uint32_t i = 0; i < G.n_term; ++i) {
    const ClauseDev &c = G.term[i];
    const int32_t v = term_value(R, C, c.lhs);
    switch (c.cmp) {
      case OCTAX_CMP_EQ: hit |= v == c.rhs; break;
      case OCTAX_CMP_NE: hit |= v != c.rhs; break;
      case OCTAX_CMP_GE: hit |= v >= c.rhs; break;
      case OCTAX_CMP_GT: hit |= v > c.rhs; break;
      case OCTAX_CMP_LE: hit |= v <= c.rhs; break;
      case OCTAX_CMP_LT: hit |= v < c.rhs; break;
      default: break;
    }
  }
  return hit;
}

// Power-on state + the game's startup instructions (no key, timers tick every
// K), then the no-op reset wrapper (§3.2): a drawn number of no-key env steps
// of frameskip frames each, unobserved. The previous action becomes the no-op.
// kWrap = false compiles the wrapper out (no game of the launch uses it).
template <bool kWrap, bool kS, bool kW>
__device__ __forceinline__ void reset_instance(Regs &R, const Ctx &C, const GameDev &G, uint32_t quirks) {
#pragma unroll
  for (int i = 0; i < 16; ++i) C.V[i * C.J] = 0;
  R.pc = 0x200;
  R.I = 0;
  R.sp = 0;
  R.dt = 0;
  R.st = 0;
  R.dirty = 0;
  R.wrange = kNoWrites;
#pragma unroll
  for (int i = 0; i < 16; ++i) C.stack[i * C.J] = 0;
#pragma unroll 8
  for (int r = 0; r < Disp<kS>::kWords; ++r) C.disp[r * C.J] = 0ull;
  R.hires = 0;  // SCHIP: every episode starts in lores with clear flag registers
  if (kS)
    for (int i = 0; i < 16; ++i) C.rpl[i] = 0;
  // Startup: full chunks of K (each followed by a tick), then the remainder
  // (no tick); after it, the no-op frames (K instructions and a tick each).
  // One loop, so that the interpreter is inlined here only once.
  const uint32_t noop_frames =
      !kWrap || G.max_noops == 0u ? 0u
                        : philox_w0(R.uid, R.env_steps, 0u, 3u, R.key0, R.key1) % (G.max_noops + 1u) * G.frameskip;
  const uint32_t full = G.startup / G.K, rem = G.startup - full * G.K;
  const uint32_t chunks = full + (rem != 0u) + noop_frames;
  R.phase = 1;
  R.draws = 0;
  for (uint32_t i = 0; i < chunks; ++i) {
    const bool partial = i == full && rem != 0u;
    run_instrs<kS, kW>(R, C, -1, quirks, partial ? rem : G.K);
    if (!partial) tick(R);
  }
  R.last_act = G.n_actions;
  R.phase = 0;
  R.draws = 0;
}

// 4 pixels (bits 0..3) -> 4 bytes of value 0/1 (byte j = bit j).
__device__ __forceinline__ uint32_t spread4(uint32_t nib) { return (nib * 0x00204081u) & 0x01010101u; }

// Pixels 16q..16q+15 of a packed row -> 16 bytes of 0/1, through a
// per-CTA table that maps a byte of pixels to its 8 output bytes.
__device__ __forceinline__ uint4 expand16(uint64_t row, uint32_t q, const uint2 *lut) {
  const uint32_t bits = (uint32_t)(row >> (16u * q)) & 0xFFFFu;
  const uint2 lo = lut[bits & 0xFFu], hi = lut[bits >> 8];
  return make_uint4(lo.x, lo.y, hi.x, hi.y);
}

// Whole-warp frame write: lane -> instance 8m + lane/4 of the warp, quarter
// lane%4 of every row, for the warp's `ipw` instances. frame (per lane, 0 =
// skip) points at the 2 KB frame of that lane's own instance.
template <bool kS>
__device__ __forceinline__ void capture_frame(const uint64_t *disp_warp, int J, uint8_t *frame,
                                              int lane, int ipw, const uint2 *lut);

// CHIP-8 frame (32 rows x 64 bytes): lanes 4i..4i+3 write the four 16-pixel
// quarters of one row of instance i (8 instances per pass).
template <>
__device__ __forceinline__ void capture_frame<false>(const uint64_t *disp_warp, int J, uint8_t *frame,
                                                     int lane, int ipw, const uint2 *lut) {
  const uint64_t mine = reinterpret_cast<uint64_t>(frame);
  const uint32_t q = lane & 3;
  const int passes = (ipw + 7) >> 3;
  for (int m = 0; m < passes; ++m) {
    const int src = 8 * m + (lane >> 2);
    const uint64_t base = __shfl_sync(kFull, mine, src);
    if (base) {
      const uint64_t *col = disp_warp + src;
      uint8_t *dst = reinterpret_cast<uint8_t *>(base) + q * 16u;
#pragma unroll 8
      for (int r = 0; r < 32; ++r) __stcs(reinterpret_cast<uint4 *>(dst + r * 64), expand16(col[r * J], q, lut));
    }
  }
}

// SCHIP frame (64 rows x 128 bytes): lanes 8i..8i+7 write the eight 16-pixel
// chunks of one row of instance i (4 instances per pass).
template <>
__device__ __forceinline__ void capture_frame<true>(const uint64_t *disp_warp, int J, uint8_t *frame,
                                                    int lane, int ipw, const uint2 *lut) {
  const uint64_t mine = reinterpret_cast<uint64_t>(frame);
  const uint32_t q = lane & 7, h = q >> 2;
  const int passes = (ipw + 3) >> 2;
  for (int m = 0; m < passes; ++m) {
    const int src = 4 * m + (lane >> 3);
    const uint64_t base = __shfl_sync(kFull, mine, src);
    if (base) {
      const uint64_t *col = disp_warp + src;
      uint8_t *dst = reinterpret_cast<uint8_t *>(base) + q * 16u;
#pragma unroll 8
      for (int r = 0; r < 64; ++r)
        __stcs(reinterpret_cast<uint4 *>(dst + r * 128), expand16(col[(2 * r + h) * J], q & 3u, lut));
    }
  }
}

// Packed frame of every instance of the warp with a non-null `frame`: its
// display words copied as they are, two per 16-byte streaming store
// (CHIP-8: 16 stores per instance, two instances per pass; SCHIP: 64).
template <bool kS>
__device__ __forceinline__ void capture_packed(const uint64_t *disp_warp, int J, uint8_t *frame, int lane,
                                               int ipw) {
  constexpr int kPairs = Disp<kS>::kWords / 2;  // 16-byte stores per instance-frame
  constexpr int kPerPass = 32 / (kPairs < 32 ? kPairs : 32);
  const uint64_t mine = reinterpret_cast<uint64_t>(frame);
  for (int m = 0; m < ipw; m += kPerPass) {
    const int src = m + lane / (32 / kPerPass);
    const uint64_t base = __shfl_sync(kFull, mine, src < 32 ? src : 31);
    if (src < ipw && base) {
      const uint64_t *col = disp_warp + src;
      for (int c = lane % (32 / kPerPass); c < kPairs; c += 32 / kPerPass) {
        const uint64_t w0 = col[(2 * c) * J], w1 = col[(2 * c + 1) * J];
        __stcs(reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(base) + c * 16),
               make_uint4((uint32_t)w0, (uint32_t)(w0 >> 32), (uint32_t)w1, (uint32_t)(w1 >> 32)));
      }
    }
  }
}

// Packed reset observation of the instances in `which` (every stack slot).
template <bool kS>
__device__ __forceinline__ void write_reset_packed(const uint64_t *disp_warp, int J, uint8_t *obs, int S,
                                                   unsigned which, int lane) {
  constexpr int kPairs = Disp<kS>::kWords / 2;
  const uint64_t mine = reinterpret_cast<uint64_t>(obs);
  while (which) {
    const int src = __ffs(which) - 1;
    which &= which - 1;
    const uint64_t base = __shfl_sync(kFull, mine, src);
    const uint64_t *col = disp_warp + src;
    for (int c = lane; c < kPairs; c += 32) {
      const uint64_t w0 = col[(2 * c) * J], w1 = col[(2 * c + 1) * J];
      const uint4 o = make_uint4((uint32_t)w0, (uint32_t)(w0 >> 32), (uint32_t)w1, (uint32_t)(w1 >> 32));
      for (int s = 0; s < S; ++s)
        __stcs(reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(base) + s * 8 * Disp<kS>::kWords + c * 16), o);
    }
  }
}

// Reset observation of the instances in `which`: the display in every stack slot.
template <bool kS>
__device__ __forceinline__ void write_reset_obs(const uint64_t *disp_warp, int J, uint8_t *obs, int S,
                                                unsigned which, int lane, const uint2 *lut) {
  const uint64_t mine = reinterpret_cast<uint64_t>(obs);
  constexpr int kChunks = Disp<kS>::kFrame / 16;  // 16-byte chunks per frame
  while (which) {
    const int src = __ffs(which) - 1;
    which &= which - 1;
    const uint64_t base = __shfl_sync(kFull, mine, src);
    const uint64_t *col = disp_warp + src;
#pragma unroll
    for (int it = 0; it < kChunks / 32; ++it) {
      const int c = it * 32 + lane;  // 16-byte chunk of the frame
      uint4 o;
      if (kS) o = expand16(col[(2 * (c >> 3) + ((c >> 2) & 1)) * J], c & 3, lut);
      else o = expand16(col[(c >> 2) * J], c & 3, lut);
      for (int s = 0; s < S; ++s)
        __stcs(reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(base) + s * Disp<kS>::kFrame + c * 16), o);
    }
  }
}

struct Smem {
  uint8_t *img;
  GameDev *game;
  void *uops;       // micro-op table (fetch_uop)
  int4 *alu;        // 8XYN coefficients (execute)
  uint2 *lut;       // byte of pixels -> 8 bytes of 0/1
  uint64_t *disp;
  uint32_t *stack;
  uint32_t *V;
};

// Shared memory of a CTA with J instances: image | game | decoded opcodes |
// expansion table | 8XYN coefficients | display [W][J] u64 | stack [16][J] u32 | V [16][J] u32,
// W = 32 (CHIP-8) or 128 (SCHIP).
template <bool kS, bool kW>
__device__ __forceinline__ Smem carve(uint8_t *smem, int J) {
  constexpr int kUopSmem = kW ? kUopSmemWide : kUopSmemNarrow;
  Smem s;
  s.img = smem;
  s.game = reinterpret_cast<GameDev *>(smem + kRamBytes);
  s.uops = smem + kRamBytes + kGameSmem;
  s.lut = reinterpret_cast<uint2 *>(smem + kRamBytes + kGameSmem + kUopSmem);
  s.alu = reinterpret_cast<int4 *>(smem + kRamBytes + kGameSmem + kUopSmem + kLutSmem);
  s.disp = reinterpret_cast<uint64_t *>(smem + kRamBytes + kGameSmem + kUopSmem + kLutSmem + kAluSmem);
  s.stack = reinterpret_cast<uint32_t *>(s.disp + Disp<kS>::kWords * J);
  s.V = s.stack + 16 * J;
  return s;
}

// Every thread of the CTA calls this (it contains a barrier).
template <bool kW>
__device__ __forceinline__ void stage_game(const Smem &S, const GameDev *games, const uint8_t *images,
                                           int game, uint32_t quirks, int J) {
  const uint4 *src = reinterpret_cast<const uint4 *>(images + (size_t)game * kRamBytes);
  uint4 *dst = reinterpret_cast<uint4 *>(S.img);
  for (int i = threadIdx.x; i < kRamBytes / 16; i += blockDim.x) dst[i] = src[i];
  const uint4 *gs = reinterpret_cast<const uint4 *>(games + game);
  uint4 *gd = reinterpret_cast<uint4 *>(S.game);
  for (int i = threadIdx.x; i < (int)(sizeof(GameDev) / 16); i += blockDim.x) gd[i] = gs[i];
  __syncthreads();
  for (int b = threadIdx.x; b < 256; b += blockDim.x) S.lut[b] = make_uint2(spread4(b & 15u), spread4(b >> 4));
  if (threadIdx.x < 16) {
    // per N: {c0, c1, c2, c3} {a, b, k, 0} (see execute); other N are never fast
    int4 r = make_int4(0, 0, 0, 0), f = make_int4(0, 0, 0, 0);
    switch (threadIdx.x) {
      case 0x0: r = make_int4(0, 1, 0, 0); break;                                    // VY
      case 0x1: r = make_int4(1, 1, -1, 0); break;                                   // x + y - (x & y) = x | y
      case 0x2: r = make_int4(0, 0, 1, 0); break;                                    // x & y
      case 0x3: r = make_int4(1, 1, -2, 0); break;                                   // x + y - 2 (x & y) = x ^ y
      case 0x4: r = make_int4(1, 1, 0, 0); f = make_int4(1, 0, 0, 0); break;         // carry = bit 8 of the sum
      case 0x5: r = make_int4(1, -1, 0, 0); f = make_int4(1, 0, 256, 0); break;      // NOT borrow: x - y + 256 >= 256
      case 0x6: r = make_int4(0, 0, 0, 1); f = make_int4(-512, 256, 0, 0); break;    // bit 0: 256 (x - 2 (x >> 1))
      case 0x7: r = make_int4(-1, 1, 0, 0); f = make_int4(1, 0, 256, 0); break;      // NOT borrow: y - x + 256 >= 256
      case 0xE: r = make_int4(2, 0, 0, 0); f = make_int4(1, 0, 0, 0); break;         // bit 7 shifted out = bit 8 of 2x
      default: break;
    }
    S.alu[2 * threadIdx.x] = r;
    S.alu[2 * threadIdx.x + 1] = f;
  }
  // decode the opcode at every even address of the image once
  for (int w = threadIdx.x; w < kRamBytes / 2; w += blockDim.x) {
    const uint32_t op = ((uint32_t)S.img[2 * w] << 8) | S.img[2 * w + 1];
    const uint32_t xo = ((op >> 8) & 15u) * (uint32_t)J, yo = ((op >> 4) & 15u) * (uint32_t)J;
    if (kW) static_cast<uint4 *>(S.uops)[w] = make_uint4(make_uop(op, quirks), xo, yo, op & 0xFFFu);
    else static_cast<uint2 *>(S.uops)[w] = make_uint2(make_uop(op, quirks), xo | (yo << 16));
  }
}

template <bool kS>
__device__ __forceinline__ void load_regs(Regs &R, const DevState &st, int64_t slot) {
  const uint32_t pcI = st.pcI[slot], misc = st.misc[slot];
  const int64_t n = st.n;
  R.pc = pcI & 0xFFFFu;
  R.I = pcI >> 16;
  R.sp = misc & 0xFFu;
  R.dt = (misc >> 8) & 0xFFu;
  R.st = (misc >> 16) & 0xFFu;
  R.status = misc >> 24;
  R.dirty = st.dirty[slot];
  R.wrange = st.wrange[slot];
  R.env_steps = st.env_steps[slot];
  R.key0 = st.key[slot];
  R.key1 = st.key[n + slot];
  R.uid = st.uid[slot];
  R.last_act = st.last_act[slot];
  R.hires = kS ? st.mode[slot] : 0u;
  R.draws = 0;
  R.phase = 0;
}

template <bool kS>
__device__ __forceinline__ void store_regs(const Regs &R, const DevState &st, int64_t slot) {
  st.pcI[slot] = R.pc | (R.I << 16);
  st.misc[slot] = R.sp | (R.dt << 8) | (R.st << 16) | (R.status << 24);
  st.dirty[slot] = R.dirty;
  st.env_steps[slot] = R.env_steps;
  st.last_act[slot] = (uint8_t)R.last_act;
  if (kS) st.mode[slot] = (uint8_t)R.hires;
}

// V0-VF: packed 4 per u32 in global memory, one per u32 in shared memory.
__device__ __forceinline__ void load_V(const Ctx &C, const DevState &st, int64_t slot) {
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    const uint32_t word = st.v[w * st.n + slot];
#pragma unroll
    for (int b = 0; b < 4; ++b) C.V[(4 * w + b) * C.J] = (word >> (8 * b)) & 0xFFu;
  }
}

__device__ __forceinline__ void store_V(const Ctx &C, const DevState &st, int64_t slot) {
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    uint32_t word = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) word |= C.V[(4 * w + b) * C.J] << (8 * b);
    st.v[w * st.n + slot] = word;
  }
}

template <bool kWrap, bool kS, bool kW>
__device__ void run_group(const StepLaunch &p, const Group &g, const Smem &S) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, ipw = p.ipw;
  const int J = (blockDim.x >> 5) * ipw;  // instances per CTA
  const int j = w * ipw + lane;           // this lane's instance (if lane < ipw)
  const DevState &st = p.st;
  const int64_t n = st.n;
  const GameDev &G = *S.game;
  const bool mine = lane < ipw;
  const bool active = mine && j < (int)g.count;
  const int64_t slot = (int64_t)g.slot0 + (active ? j : 0);
  const IO io = p.io_table ? p.io_table[g.io] : p.io0;
  const uint32_t quirks = p.quirks;
  uint64_t *disp_warp = S.disp + w * ipw;

  Regs R;
  load_regs<kS>(R, st, slot);
  const int64_t row = active ? (int64_t)st.out_row[slot] : 0;
  uint32_t ep = st.ep[slot];
  int32_t prev = st.prev_score[slot];
  if (mine) {
#pragma unroll
    for (int i = 0; i < 16; ++i) S.stack[i * J + j] = st.stack[i * n + slot];
#pragma unroll 8
    for (int r = 0; r < Disp<kS>::kWords; ++r) S.disp[r * J + j] = st.disp[r * n + slot];
  }
  const Ctx C{S.disp + (mine ? j : 0), S.stack + (mine ? j : 0), S.V + (mine ? j : 0),
              st.ram + slot * (int64_t)kRamBytes, J, S.uops, S.alu, st.rpl + slot * 16};
  if (mine) load_V(C, st, slot);
  const uint32_t K = G.K, FS = G.frameskip, first_kept = FS - (uint32_t)p.S;
  __syncwarp();

  for (int s = 0; s < p.steps; ++s) {
    const int64_t io_row = (int64_t)(p.step0 + s) * io.rows + row;
    int key = -1;
    uint8_t *my_obs = nullptr;
    if (active) {
      uint32_t a = io.actions[io_row];
      // sticky actions (§3.2): repeat the previous step's action with probability sticky / 2^32
      if (kWrap && G.sticky != 0u && philox_w0(R.uid, R.env_steps, 0u, 2u, R.key0, R.key1) < G.sticky) a = R.last_act;
      R.last_act = a;
      if (a < G.n_actions) key = G.action_set[a] & 15;
      else if (a > G.n_actions) R.status |= OCTAX_STATUS_BAD_ACTION;
      my_obs = io.obs + io_row * (int64_t)p.S * (io.packed ? 8 * Disp<kS>::kWords : Disp<kS>::kFrame);
    }
    R.draws = 0;
    R.phase = 0;
    for (uint32_t f = 0; f < FS; ++f) {
      if (active) {
        run_instrs<kS, kW>(R, C, key, quirks, K);
        tick(R);
      }
      if (f >= first_kept) {
        __syncwarp();
        if (io.packed)
          capture_packed<kS>(disp_warp, J, my_obs ? my_obs + (f - first_kept) * 8 * Disp<kS>::kWords : nullptr,
                             lane, ipw);
        else
          capture_frame<kS>(disp_warp, J, my_obs ? my_obs + (f - first_kept) * Disp<kS>::kFrame : nullptr, lane,
                            ipw, S.lut);
        __syncwarp();
      }
    }
    bool done = false;
    if (active) {
      const int32_t sc = score(R, C, G);
      ep += 1;
      R.env_steps += 1;
      done = terminated(R, C, G) || (G.max_steps != 0 && ep >= G.max_steps);
      io.reward[io_row] = (float)(sc - prev);
      io.done[io_row] = done ? 1 : 0;
      if (done) {
        reset_instance<kWrap, kS, kW>(R, C, G, quirks);
        ep = 0;
        prev = score(R, C, G);
      } else {
        prev = sc;
      }
    }
    const unsigned which = __ballot_sync(kFull, done);
    if (which) {
      __syncwarp();
      if (io.packed) write_reset_packed<kS>(disp_warp, J, my_obs, p.S, which, lane);
      else write_reset_obs<kS>(disp_warp, J, my_obs, p.S, which, lane, S.lut);
      __syncwarp();
    }
  }

  if (active) {
    store_regs<kS>(R, st, slot);
    store_V(C, st, slot);
    st.wrange[slot] = R.wrange;
    st.ep[slot] = ep;
    st.prev_score[slot] = prev;
#pragma unroll
    for (int i = 0; i < 16; ++i) st.stack[i * n + slot] = (uint16_t)S.stack[i * J + j];
#pragma unroll 8
    for (int r = 0; r < Disp<kS>::kWords; ++r) st.disp[r * n + slot] = S.disp[r * J + j];
  }
}

// One CTA's loop over groups (a persistent CTA pulls them off the queue).
template <bool kWrap, bool kS, bool kW>
__device__ __forceinline__ void step_body(const StepLaunch &p) {
  uint8_t *const smem = g_smem;
  const Smem S = carve<kS, kW>(smem, (blockDim.x >> 5) * p.ipw);
  __shared__ int s_group;
  int cur_game = -1;
  int gi = blockIdx.x;
  for (;;) {
    if (p.work_counter) {
      if (threadIdx.x == 0) s_group = (int)atomicAdd(p.work_counter, 1u);
      __syncthreads();
      gi = s_group;
    }
    if (gi >= p.n_groups) break;
    const Group g = p.groups[gi];
    if ((int)g.game != cur_game) {
      stage_game<kW>(S, p.games, p.images, g.game, p.quirks, (blockDim.x >> 5) * p.ipw);
      cur_game = g.game;
    }
    __syncthreads();
    run_group<kWrap, kS, kW>(p, g, S);
    __syncthreads();  // shared memory is reused by the next group
    if (!p.work_counter) break;
  }
}

// kWrap: the sticky-action / no-op-reset variant (games without the wrappers
// run the kernel without them); kS: the Super-CHIP display layout.
// kW: 16-byte micro-op table (the launcher picks it where it costs no
// occupancy; Super-CHIP kernels, whose displays dominate shared memory, use
// the 8-byte table). Every step kernel is held to 128 registers (two
// 256-thread CTAs per SM): unbounded, the wrapper and Super-CHIP
// instantiations took 157-210 and ran 12-16 % slower.
template <bool kW>
__global__ void __launch_bounds__(kMaxBlock, 2) step_kernel_chip8(const StepLaunch p) {
  step_body<false, false, kW>(p);
}

template <bool kWrap, bool kS, bool kW>
__global__ void __launch_bounds__(kMaxBlock, 2) step_kernel(const StepLaunch p) {
  step_body<kWrap, kS, kW>(p);
}


// ---------------------------------------------------------------------------
// Warp-specialised step: the first block/32 warps emulate (as in run_group),
// the last `writers` warps only write observations. At every kept frame the
// emulators copy their packed display rows into one slot of a two-slot ring
// in shared memory and go on emulating; the writers expand that slot to
// uint8 frames and stream them out, so interpreter and stores overlap. After
// each step a last message carries the done flags and reset displays; the
// writer thread that wrote an address earlier in the step is the one that
// overwrites it with the reset observation, so program order keeps them
// ordered. Slots hand over through mbarriers (full: all emulator threads
// arrive; empty: all writer threads arrive); every wait polls a bounded
// number of times for at most kMaxWaitNs of the global timer and, if it
// gives up, records the failure in p.err and stops the thread's work instead
// of hanging.

constexpr uint32_t kMaxPolls = 1u << 22;
constexpr uint64_t kMaxWaitNs = 1000000000ull;  // one second

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(b))
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, unsigned int *err) {
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0; i < kMaxPolls; ++i) {
    if (mbar_try(b, parity)) return true;
    if (global_ns() - t0 > kMaxWaitNs) break;
  }
  atomicOr(err, 1u);
  return false;
}

struct WsSmem {
  Smem base;
  uint64_t *ring;    // [2][32][J] snapshots of packed display rows
  uint8_t *done;     // [2][J] done flags of the end-of-step message
  uint64_t *full;    // [2]
  uint64_t *empty;   // [2]
};

// base layout | ring | done flags | barriers
__device__ __forceinline__ WsSmem carve_ws(uint8_t *smem, int J) {
  WsSmem w;
  w.base = carve<false, false>(smem, J);
  w.ring = reinterpret_cast<uint64_t *>(w.base.V + 16 * J);
  w.done = reinterpret_cast<uint8_t *>(w.ring + 2 * 32 * J);
  w.full = reinterpret_cast<uint64_t *>(w.done + ((2 * J + 15) & ~15));
  w.empty = w.full + 2;
  return w;
}

// Emulator side of one group. `msg` counts messages of this CTA.
__device__ void run_group_emu(const StepLaunch &p, const Group &g, const WsSmem &W, uint32_t &msg,
                              bool &failed) {
  const Smem &S = W.base;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, ipw = p.ipw;
  const int E = (int)(blockDim.x >> 5) - p.writers;
  const int J = E * ipw;
  const int j = w * ipw + lane;
  const DevState &st = p.st;
  const int64_t n = st.n;
  const GameDev &G = *S.game;
  const bool mine = lane < ipw;
  const bool active = mine && j < (int)g.count;
  const int64_t slot = (int64_t)g.slot0 + (active ? j : 0);
  const IO io = p.io_table ? p.io_table[g.io] : p.io0;
  const uint32_t quirks = p.quirks;

  Regs R;
  load_regs<false>(R, st, slot);
  const int64_t row = active ? (int64_t)st.out_row[slot] : 0;
  uint32_t ep = st.ep[slot];
  int32_t prev = st.prev_score[slot];
  if (mine) {
#pragma unroll
    for (int i = 0; i < 16; ++i) S.stack[i * J + j] = st.stack[i * n + slot];
#pragma unroll 8
    for (int r = 0; r < 32; ++r) S.disp[r * J + j] = st.disp[r * n + slot];
  }
  const Ctx C{S.disp + (mine ? j : 0), S.stack + (mine ? j : 0), S.V + (mine ? j : 0),
              st.ram + slot * (int64_t)kRamBytes, J, S.uops, S.alu, st.rpl + slot * 16};
  if (mine) load_V(C, st, slot);
  const uint32_t K = G.K, FS = G.frameskip, first_kept = FS - (uint32_t)p.S;

  for (int s = 0; s < p.steps && !failed; ++s) {
    const int64_t io_row = (int64_t)(p.step0 + s) * io.rows + row;
    int key = -1;
    if (active) {
      uint32_t a = io.actions[io_row];
      // sticky actions (§3.2): repeat the previous step's action with probability sticky / 2^32
      if (G.sticky != 0u && philox_w0(R.uid, R.env_steps, 0u, 2u, R.key0, R.key1) < G.sticky) a = R.last_act;
      R.last_act = a;
      if (a < G.n_actions) key = G.action_set[a] & 15;
      else if (a > G.n_actions) R.status |= OCTAX_STATUS_BAD_ACTION;
    }
    R.draws = 0;
    R.phase = 0;
    for (uint32_t f = 0; f < FS && !failed; ++f) {
      if (active) {
        run_instrs<false, false>(R, C, key, quirks, K);
        tick(R);
      }
      if (f >= first_kept) {  // hand the frame to the writers
        const uint32_t b = msg & 1u, use = msg >> 1;
        if (!mbar_wait(W.empty + b, (use & 1u) ^ 1u, p.err)) {
          failed = true;
          break;
        }
        if (mine) {
          uint64_t *dst = W.ring + b * 32 * J + j;
#pragma unroll 8
          for (int r = 0; r < 32; ++r) dst[r * J] = S.disp[r * J + j];
        }
        mbar_arrive(W.full + b);
        ++msg;
      }
    }
    if (failed) break;
    bool done = false;
    if (active) {
      const int32_t sc = score(R, C, G);
      ep += 1;
      R.env_steps += 1;
      done = terminated(R, C, G) || (G.max_steps != 0 && ep >= G.max_steps);
      io.reward[io_row] = (float)(sc - prev);
      io.done[io_row] = done ? 1 : 0;
      if (done) {
        reset_instance<true, false, false>(R, C, G, quirks);
        ep = 0;
        prev = score(R, C, G);
      } else {
        prev = sc;
      }
    }
    // end-of-step message: done flags and the reset displays
    const uint32_t b = msg & 1u, use = msg >> 1;
    if (!mbar_wait(W.empty + b, (use & 1u) ^ 1u, p.err)) {
      failed = true;
      break;
    }
    if (mine) {
      W.done[b * J + j] = done ? 1 : 0;
      if (done) {
        uint64_t *dst = W.ring + b * 32 * J + j;
#pragma unroll 8
        for (int r = 0; r < 32; ++r) dst[r * J] = S.disp[r * J + j];
      }
    }
    mbar_arrive(W.full + b);
    ++msg;
  }

  if (active && !failed) {
    store_regs<false>(R, st, slot);
    store_V(C, st, slot);
    st.wrange[slot] = R.wrange;
    st.ep[slot] = ep;
    st.prev_score[slot] = prev;
#pragma unroll
    for (int i = 0; i < 16; ++i) st.stack[i * n + slot] = (uint16_t)S.stack[i * J + j];
#pragma unroll 8
    for (int r = 0; r < 32; ++r) st.disp[r * n + slot] = S.disp[r * J + j];
  }
}

// Writer side of one group: writer warp ww owns instances
// [ww * J/W, (ww + 1) * J/W); lane -> instance 8m + lane/4, quarter lane%4.
__device__ void run_group_writer(const StepLaunch &p, const Group &g, const WsSmem &W, uint32_t &msg,
                                 bool &failed) {
  if (p.stall_writers) return;  // diagnostic: never hand slots back (see octax_debug_stall_writers)
  const int t = threadIdx.x, lane = t & 31;
  const int E = (int)(blockDim.x >> 5) - p.writers;
  const int J = E * p.ipw;
  const int per = J / p.writers, passes = per >> 3;  // per in {8, 16, 32}
  const int ww = (t >> 5) - E;
  const uint32_t q = lane & 3u;
  const IO io = p.io_table ? p.io_table[g.io] : p.io0;
  const int S_ = p.S;
  int jj[4];
  int64_t orow[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    jj[m] = ww * per + 8 * m + (lane >> 2);
    const bool act = m < passes && jj[m] < (int)g.count;
    orow[m] = act ? (int64_t)p.st.out_row[(int64_t)g.slot0 + jj[m]] : -1;
  }
  const GameDev &G = *W.base.game;
  const uint32_t FS = G.frameskip, first_kept = FS - (uint32_t)S_;
  for (int s = 0; s < p.steps && !failed; ++s) {
    const int64_t step_row = (int64_t)(p.step0 + s) * io.rows;
    for (uint32_t f = first_kept; f <= FS; ++f) {  // FS - S frames, then the end-of-step message
      const uint32_t b = msg & 1u, use = msg >> 1;
      if (!mbar_wait(W.full + b, use & 1u, p.err)) {
        failed = true;
        break;
      }
      const uint64_t *ring = W.ring + b * 32 * J;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        if (m >= passes || orow[m] < 0) continue;
        uint8_t *obs = io.obs + (step_row + orow[m]) * (int64_t)S_ * kFrameBytes + q * 16u;
        const uint64_t *col = ring + jj[m];
        if (f < FS) {
          uint8_t *dst = obs + (f - first_kept) * kFrameBytes;
#pragma unroll 8
          for (int r = 0; r < 32; ++r)
            __stcs(reinterpret_cast<uint4 *>(dst + r * 64), expand16(col[r * J], q, W.base.lut));
        } else if (W.done[b * J + jj[m]]) {
          for (int r = 0; r < 32; ++r) {
            const uint4 o = expand16(col[r * J], q, W.base.lut);
            for (int k = 0; k < S_; ++k)
              __stcs(reinterpret_cast<uint4 *>(obs + k * kFrameBytes + r * 64), o);
          }
        }
      }
      mbar_arrive(W.empty + b);
      ++msg;
    }
  }
}

__global__ void step_kernel_ws(const StepLaunch p) {
  uint8_t *const smem = g_smem;
  const int E = (int)(blockDim.x >> 5) - p.writers;
  const int J = E * p.ipw;
  const WsSmem W = carve_ws(smem, J);
  __shared__ int s_group;
  if (threadIdx.x == 0) {
    mbar_init(W.full + 0, (uint32_t)E * 32u);
    mbar_init(W.full + 1, (uint32_t)E * 32u);
    mbar_init(W.empty + 0, (uint32_t)p.writers * 32u);
    mbar_init(W.empty + 1, (uint32_t)p.writers * 32u);
  }
  __syncthreads();
  const bool writer = (int)(threadIdx.x >> 5) >= E;
  uint32_t msg = 0;
  bool failed = false;
  int cur_game = -1;
  int gi = blockIdx.x;
  for (;;) {
    if (p.work_counter) {
      if (threadIdx.x == 0) s_group = (int)atomicAdd(p.work_counter, 1u);
      __syncthreads();
      gi = s_group;
    }
    if (gi >= p.n_groups) break;
    const Group g = p.groups[gi];
    if ((int)g.game != cur_game) {
      stage_game<false>(W.base, p.games, p.images, g.game, p.quirks, J);
      cur_game = g.game;
    }
    __syncthreads();
    if (!failed) {
      if (writer) run_group_writer(p, g, W, msg, failed);
      else run_group_emu(p, g, W, msg, failed);
    }
    __syncthreads();  // shared memory is reused by the next group
    if (!p.work_counter) break;
  }
}

template <bool kS>
__global__ void __launch_bounds__(kMaxBlock) reset_kernel(const ResetLaunch p) {
  uint8_t *const smem = g_smem;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, ipw = p.ipw;
  const int J = (blockDim.x >> 5) * ipw;
  const int j = w * ipw + lane;
  const Smem S = carve<kS, false>(smem, J);
  const Group g = p.groups[blockIdx.x];
  stage_game<false>(S, p.games, p.images, g.game, p.quirks, J);
  __syncthreads();
  const DevState &st = p.st;
  const int64_t n = st.n;
  const GameDev &G = *S.game;
  const bool mine = lane < ipw;
  const bool active = mine && j < (int)g.count;
  const int64_t slot = (int64_t)g.slot0 + (active ? j : 0);
  const int64_t row = !active ? 0 : (p.init && p.set_rows) ? (int64_t)(g.row0 + j) : (int64_t)st.out_row[slot];
  const bool doit = active && (p.mask == nullptr || p.mask[row] != 0);
  Regs R;
  if (p.init) {
    const uint64_t seed = p.seed_of_group ? p.seed_of_group[blockIdx.x] : p.seed;
    R.status = 0;
    R.env_steps = 0;
    R.key0 = (uint32_t)(seed & 0xFFFFFFFFu);
    R.key1 = (uint32_t)(seed >> 32);
    R.uid = p.uid_of_slot ? p.uid_of_slot[slot] : (uint32_t)row;
  } else {
    load_regs<kS>(R, st, slot);
  }
  const Ctx C{S.disp + (mine ? j : 0), S.stack + (mine ? j : 0), S.V + (mine ? j : 0),
              st.ram + slot * (int64_t)kRamBytes, J, S.uops, S.alu, st.rpl + slot * 16};
  if (doit) reset_instance<true, kS, false>(R, C, G, p.quirks);
  const unsigned which = __ballot_sync(kFull, doit);
  if (p.obs && which) {
    __syncwarp();
    write_reset_obs<kS>(S.disp + w * ipw, J, doit ? p.obs + row * (int64_t)p.S * Disp<kS>::kFrame : nullptr,
                        p.S, which, lane, S.lut);
    __syncwarp();
  }
  if (doit) {
    store_regs<kS>(R, st, slot);
    store_V(C, st, slot);
    st.wrange[slot] = R.wrange;
    st.ep[slot] = 0;
    st.prev_score[slot] = score(R, C, G);
    if (p.init) {
      st.key[slot] = R.key0;
      st.key[n + slot] = R.key1;
      st.uid[slot] = R.uid;
      if (p.set_rows) {
        st.out_row[slot] = (uint32_t)row;
        st.game[slot] = g.game;
      }
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) st.stack[i * n + slot] = (uint16_t)S.stack[i * J + j];
#pragma unroll 8
    for (int r = 0; r < Disp<kS>::kWords; ++r) st.disp[r * n + slot] = S.disp[r * J + j];
  }
}

// RAM byte of a slot as the program sees it.
__device__ __forceinline__ uint8_t ram_byte(const DevState &st, const uint8_t *img, int64_t slot,
                                            uint64_t dirty, uint32_t a) {
  return ((dirty >> (a >> kPageShift)) & 1u) ? st.ram[slot * (int64_t)kRamBytes + a] : img[a];
}

__device__ __forceinline__ uint64_t fnv_byte(uint64_t h, uint32_t b) {
  return (h ^ (uint64_t)(b & 0xFFu)) * 1099511628211ull;
}

__global__ void hash_kernel(const DevState st, const uint8_t *images, const uint32_t *slot_of_row,
                            int64_t rows, uint64_t *out) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= rows) return;
  const int64_t slot = slot_of_row[row];
  const int64_t n = st.n;
  const uint8_t *img = images + (size_t)st.game[slot] * kRamBytes;
  uint64_t h = 14695981039346656037ull;
  for (int j = 0; j < 4; ++j) {
    const uint32_t w = st.v[j * n + slot];
    for (int b = 0; b < 4; ++b) h = fnv_byte(h, w >> (8 * b));
  }
  const uint32_t pcI = st.pcI[slot], misc = st.misc[slot];
  const uint32_t I = pcI >> 16, PC = pcI & 0xFFFFu;
  h = fnv_byte(h, I);
  h = fnv_byte(h, I >> 8);
  h = fnv_byte(h, PC);
  h = fnv_byte(h, PC >> 8);
  for (int b = 0; b < 4; ++b) h = fnv_byte(h, misc >> (8 * b));  // SP DT ST status
  for (int i = 0; i < 16; ++i) {
    const uint32_t e = st.stack[i * n + slot];
    h = fnv_byte(h, e);
    h = fnv_byte(h, e >> 8);
  }
  for (int r = 0; r < disp_words(st.schip); ++r) {  // SCHIP words run [y][h], as in the record
    const uint64_t w = st.disp[r * n + slot];
    for (int b = 0; b < 8; ++b) h = fnv_byte(h, (uint32_t)(w >> (8 * b)));
  }
  const uint64_t dirty = st.dirty[slot];
  for (uint32_t a = 0; a < (uint32_t)kRamBytes; ++a) h = fnv_byte(h, ram_byte(st, img, slot, dirty, a));
  const uint32_t ep = st.ep[slot], es = st.env_steps[slot];
  for (int b = 0; b < 4; ++b) h = fnv_byte(h, ep >> (8 * b));
  for (int b = 0; b < 4; ++b) h = fnv_byte(h, es >> (8 * b));
  h = fnv_byte(h, st.last_act[slot]);
  if (st.schip) {
    h = fnv_byte(h, st.mode[slot]);
    for (int i = 0; i < 16; ++i) h = fnv_byte(h, st.rpl[slot * 16 + i]);
  }
  out[row] = h;
}

__global__ void records_kernel(const DevState st, const uint8_t *images, const uint32_t *slot_of_row,
                               int64_t first, int64_t count, octax_state_record *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int64_t slot = slot_of_row[first + i];
  const int64_t n = st.n;
  octax_state_record &rec = out[i];
  for (int j = 0; j < 4; ++j) {
    const uint32_t w = st.v[j * n + slot];
    for (int b = 0; b < 4; ++b) rec.V[4 * j + b] = (uint8_t)(w >> (8 * b));
  }
  const uint32_t pcI = st.pcI[slot], misc = st.misc[slot];
  rec.PC = (uint16_t)(pcI & 0xFFFFu);
  rec.I = (uint16_t)(pcI >> 16);
  rec.SP = (uint8_t)misc;
  rec.DT = (uint8_t)(misc >> 8);
  rec.ST = (uint8_t)(misc >> 16);
  rec.status = (uint8_t)(misc >> 24);
  for (int k = 0; k < 16; ++k) rec.stack[k] = st.stack[k * n + slot];
  for (int y = 0; y < 64; ++y)
    for (int hw = 0; hw < 2; ++hw)
      rec.display[y][hw] = st.schip ? st.disp[(2 * y + hw) * n + slot]
                                    : (y < 32 && hw == 0 ? st.disp[y * n + slot] : 0ull);
  const uint8_t *img = images + (size_t)st.game[slot] * kRamBytes;
  const uint64_t dirty = st.dirty[slot];
  for (uint32_t a = 0; a < (uint32_t)kRamBytes; ++a) rec.ram[a] = ram_byte(st, img, slot, dirty, a);
  rec.episode_steps = st.ep[slot];
  rec.env_steps = st.env_steps[slot];
  rec.last_action = st.last_act[slot];
  rec.hires = st.schip ? st.mode[slot] : 0;
  for (int k = 0; k < 6; ++k) rec.pad[k] = 0;
  for (int k = 0; k < 16; ++k) rec.rpl[k] = st.schip ? st.rpl[slot * 16 + k] : 0;
}

__global__ void set_records_kernel(const DevState st, const GameDev *games, const uint8_t *images,
                                   const uint32_t *slot_of_row, int64_t first, int64_t count,
                                   const octax_state_record *in) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int64_t slot = slot_of_row[first + i];
  const int64_t n = st.n;
  const octax_state_record &rec = in[i];
  for (int j = 0; j < 4; ++j) {
    uint32_t w = 0;
    for (int b = 0; b < 4; ++b) w |= (uint32_t)rec.V[4 * j + b] << (8 * b);
    st.v[j * n + slot] = w;
  }
  st.pcI[slot] = (uint32_t)(rec.PC & 0xFFFu) | ((uint32_t)rec.I << 16);
  st.misc[slot] = (uint32_t)rec.SP | ((uint32_t)rec.DT << 8) | ((uint32_t)rec.ST << 16) |
                  ((uint32_t)rec.status << 24);
  for (int k = 0; k < 16; ++k) st.stack[k * n + slot] = rec.stack[k];
  for (int r = 0; r < disp_words(st.schip); ++r)
    st.disp[r * n + slot] = st.schip ? rec.display[r >> 1][r & 1] : rec.display[r][0];
  st.mode[slot] = st.schip ? rec.hires : 0;
  for (int k = 0; k < 16; ++k) st.rpl[slot * 16 + k] = st.schip ? rec.rpl[k] : 0;
  const int game = st.game[slot];
  const uint8_t *img = images + (size_t)game * kRamBytes;
  uint64_t dirty = 0;
  uint32_t lo = 0xFFFu, hi = 0u;
  uint8_t *ram = st.ram + slot * (int64_t)kRamBytes;
  for (int page = 0; page < kRamBytes >> kPageShift; ++page) {
    bool differs = false;
    for (int b = 0; b < (1 << kPageShift); ++b) {
      const int a = (page << kPageShift) + b;
      if (rec.ram[a] != img[a]) {
        differs = true;
        lo = a < (int)lo ? (uint32_t)a : lo;
        hi = (uint32_t)a;
      }
    }
    if (differs) {
      dirty |= 1ull << page;
      for (int b = 0; b < (1 << kPageShift); ++b) ram[(page << kPageShift) + b] = rec.ram[(page << kPageShift) + b];
    }
  }
  st.dirty[slot] = dirty;
  st.wrange[slot] = lo | hi << 16;  // the bytes that differ from the image lie in [lo, hi]
  st.ep[slot] = rec.episode_steps;
  st.env_steps[slot] = rec.env_steps;
  st.last_act[slot] = rec.last_action;
  // score of the restored state (the next step's reward baseline)
  const GameDev &G = games[game];
  int32_t s = 0;
  for (uint32_t k = 0; k < G.n_score; ++k) {
    const TermDev &t = G.score[k];
    const int32_t v = t.src == OCTAX_SRC_REG ? (int32_t)rec.V[t.idx & 15] : (int32_t)rec.ram[t.idx & 0xFFF];
    switch (t.xform) {
      case OCTAX_X_RAW: s += v; break;
      case OCTAX_X_NEG: s -= v; break;
      case OCTAX_X_DEC_TENS: s += v / 10; break;
      case OCTAX_X_DEC_ONES: s += v % 10; break;
      case OCTAX_X_DEC_TENS_MINUS_ONES: s += v / 10 - v % 10; break;
      case OCTAX_X_NIB_HI_MINUS_LO: s += (v >> 4) - (v & 15); break;
      case OCTAX_X_ZERO_IF_GT: s += v > t.arg ? 0 : v; break;
      default: break;
    }
  }
  st.prev_score[slot] = s;
}

}  // namespace

size_t step_smem_bytes(int block, int ipw, int schip, int wide) {
  const size_t J = (size_t)(block / 32) * ipw;
  return (size_t)kRamBytes + kGameSmem + (wide ? kUopSmemWide : kUopSmemNarrow) + kLutSmem + kAluSmem +
         J * (disp_words(schip) * sizeof(uint64_t) + 32 * sizeof(uint32_t));
}

// Dynamic shared memory a CTA may opt into, less room for static shared data.
// Opt-in dynamic shared memory limit of the current device (less 1 KB for
// static shared memory), queried once per device ordinal.
size_t max_dynamic_smem() {
  static std::mutex mu;
  static std::map<int, size_t> per_dev;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = per_dev.find(dev);
  if (it != per_dev.end()) return it->second;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || optin <= 0)
    optin = 99 * 1024;
  const size_t v = (size_t)optin - 1024;
  per_dev[dev] = v;
  return v;
}

size_t step_ws_smem_bytes(int block, int ipw) {
  const size_t J = (size_t)(block / 32) * ipw;
  return step_smem_bytes(block, ipw, 0) + 2 * 32 * 8 * J + ((2 * J + 15) & ~(size_t)15) + 4 * 8;
}

// The dynamic shared memory attribute of a kernel applies to the current
// device only, so it is set once per device ordinal (under a lock: the
// serving thread and user threads launch concurrently).
static cudaError_t ensure_smem_attr() {
  static std::mutex mu;
  static std::map<int, bool> done;
  int dev = 0;
  cudaError_t de = cudaGetDevice(&dev);
  if (de != cudaSuccess) return de;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return cudaSuccess;
  const size_t cap = max_dynamic_smem();
  auto lim = [&](int schip, int wide) { return (int)std::min(step_smem_bytes(kMaxBlock, 32, schip, wide), cap); };
  const struct {
    const void *fn;
    int smem;
  } fns[] = {
      {(const void *)step_kernel_chip8<true>, lim(0, 1)},       {(const void *)step_kernel_chip8<false>, lim(0, 0)},
      {(const void *)step_kernel<true, false, true>, lim(0, 1)}, {(const void *)step_kernel<true, false, false>, lim(0, 0)},
      {(const void *)step_kernel<false, true, false>, lim(1, 0)}, {(const void *)step_kernel<true, true, false>, lim(1, 0)},
      {(const void *)reset_kernel<false>, lim(0, 0)},            {(const void *)reset_kernel<true>, lim(1, 0)},
      {(const void *)step_kernel_ws, (int)cap}};
  for (const auto &f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, f.smem);
    if (e != cudaSuccess) return e;
  }
  done[dev] = true;
  return cudaSuccess;
}

// CHIP-8 step kernel (no writer warps) for a shape: the 16-byte micro-op
// table when it fits and keeps the narrow table's resident CTAs per SM.
static bool use_wide(int block, int ipw, int wrappers) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int>, bool> memo;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_tuple(dev, block, ipw, wrappers);
  auto it = memo.find(key);
  if (it != memo.end()) return it->second;
  const size_t sw = step_smem_bytes(block, ipw, 0, 1), sn = step_smem_bytes(block, ipw, 0, 0);
  bool wide = false;
  if (sw <= max_dynamic_smem()) {
    int ow = 0, on = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &ow, wrappers ? (const void *)step_kernel<true, false, true> : (const void *)step_kernel_chip8<true>, block, sw);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &on, wrappers ? (const void *)step_kernel<true, false, false> : (const void *)step_kernel_chip8<false>, block, sn);
    wide = ow >= on && ow > 0;
  }
  memo[key] = wide;
  return wide;
}

// The step kernel instantiation for a launch (null: writer warps on SCHIP).
static const void *step_fn(const StepLaunch &p, int block) {
  if (p.writers > 0) return p.st.schip ? nullptr : (const void *)step_kernel_ws;
  if (p.st.schip)
    return p.wrappers ? (const void *)step_kernel<true, true, false> : (const void *)step_kernel<false, true, false>;
  if (use_wide(block, p.ipw, p.wrappers))
    return p.wrappers ? (const void *)step_kernel<true, false, true> : (const void *)step_kernel_chip8<true>;
  return p.wrappers ? (const void *)step_kernel<true, false, false> : (const void *)step_kernel_chip8<false>;
}

static size_t step_fn_smem(const StepLaunch &p, int block) {
  if (p.writers > 0) return step_ws_smem_bytes(block, p.ipw);
  const int wide = !p.st.schip && use_wide(block, p.ipw, p.wrappers);
  return step_smem_bytes(block, p.ipw, p.st.schip, wide);
}

cudaError_t launch_step(const StepLaunch &p, int grid, int block, cudaStream_t s) {
  if (!state_complete(p.st)) return cudaErrorInvalidValue;
  cudaError_t e = ensure_smem_attr();
  if (e != cudaSuccess) return e;
  if (grid <= 0) return cudaSuccess;
  const void *fn = step_fn(p, block);
  if (!fn) return cudaErrorInvalidValue;
  StepLaunch copy = p;
  void *args[] = {&copy};
  const int threads = p.writers > 0 ? block + 32 * p.writers : block;
  return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3((unsigned)threads), args, step_fn_smem(p, block), s);
}

cudaError_t launch_reset(const ResetLaunch &p, int block, cudaStream_t s) {
  if (!state_complete(p.st)) return cudaErrorInvalidValue;
  cudaError_t e = ensure_smem_attr();
  if (e != cudaSuccess) return e;
  if (p.n_groups <= 0) return cudaSuccess;
  if (p.st.schip)
    reset_kernel<true><<<p.n_groups, block, step_smem_bytes(block, p.ipw, 1), s>>>(p);
  else
    reset_kernel<false><<<p.n_groups, block, step_smem_bytes(block, p.ipw, 0), s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_hash(const DevState &st, const uint8_t *images, const uint32_t *slot_of_row,
                        int64_t rows, uint64_t *out, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  if (!state_complete(st)) return cudaErrorInvalidValue;
  const int tb = 128;
  hash_kernel<<<(unsigned)((rows + tb - 1) / tb), tb, 0, s>>>(st, images, slot_of_row, rows, out);
  return cudaGetLastError();
}

cudaError_t launch_records(const DevState &st, const uint8_t *images, const uint32_t *slot_of_row,
                           int64_t first, int64_t count, octax_state_record *out, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (!state_complete(st)) return cudaErrorInvalidValue;
  const int tb = 128;
  records_kernel<<<(unsigned)((count + tb - 1) / tb), tb, 0, s>>>(st, images, slot_of_row, first, count,
                                                                   out);
  return cudaGetLastError();
}

cudaError_t launch_set_records(const DevState &st, const GameDev *games, const uint8_t *images,
                               const uint32_t *slot_of_row, int64_t first, int64_t count,
                               const octax_state_record *in, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (!state_complete(st)) return cudaErrorInvalidValue;
  const int tb = 128;
  set_records_kernel<<<(unsigned)((count + tb - 1) / tb), tb, 0, s>>>(st, games, images, slot_of_row,
                                                                       first, count, in);
  return cudaGetLastError();
}

cudaError_t add_step_node(cudaGraph_t g, cudaGraphNode_t *node, cudaGraphNode_t dep, const StepLaunch &p,
                          int grid, int block) {
  if (!state_complete(p.st)) return cudaErrorInvalidValue;
  cudaError_t e = ensure_smem_attr();
  if (e != cudaSuccess) return e;
  const void *fn = step_fn(p, block);
  if (!fn) return cudaErrorInvalidValue;
  StepLaunch copy = p;
  void *args[] = {&copy};
  cudaKernelNodeParams kp;
  memset(&kp, 0, sizeof kp);
  kp.func = const_cast<void *>(fn);
  kp.gridDim = dim3((unsigned)grid);
  kp.blockDim = dim3((unsigned)(p.writers > 0 ? block + 32 * p.writers : block));
  kp.sharedMemBytes = (unsigned)step_fn_smem(p, block);
  kp.kernelParams = args;
  return cudaGraphAddKernelNode(node, g, dep ? &dep : nullptr, dep ? 1 : 0, &kp);
}

cudaError_t alloc_state(DevState &st, int64_t n, int schip, void **block_out, size_t *bytes_out) {
  const size_t N = (size_t)n;
  // every array starts on a 256-byte boundary
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t sizes[] = {16 * N, 4 * N, 4 * N, 32 * N, 8 * (size_t)disp_words(schip) * N, 8 * N, 4096 * N,
                          4 * N,  4 * N, 4 * N, 8 * N,  4 * N,   4 * N, 2 * N, N, N, 16 * N, 4 * N};
  size_t total = 0;
  for (size_t b : sizes) total += up(b);
  uint8_t *base = nullptr;
  cudaError_t e = cudaMalloc(&base, total);
  if (e != cudaSuccess) return e;
  size_t off = 0;
  void **dst[] = {(void **)&st.v,   (void **)&st.pcI,        (void **)&st.misc,      (void **)&st.stack,
                  (void **)&st.disp, (void **)&st.dirty,     (void **)&st.ram,       (void **)&st.ep,
                  (void **)&st.env_steps, (void **)&st.prev_score, (void **)&st.key, (void **)&st.uid,
                  (void **)&st.out_row, (void **)&st.game, (void **)&st.last_act, (void **)&st.mode,
                  (void **)&st.rpl, (void **)&st.wrange};
  for (int i = 0; i < 18; ++i) {
    *dst[i] = base + off;
    off += up(sizes[i]);
  }
  st.n = n;
  st.schip = schip;
  *block_out = base;
  *bytes_out = total;
  return cudaSuccess;
}

int max_resident_ctas(int block, int ipw, int writers, int wrappers, int schip) {
  if (ensure_smem_attr() != cudaSuccess) return 0;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (writers > 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_kernel_ws, block + 32 * writers,
                                                  step_ws_smem_bytes(block, ipw));
  else {
    StepLaunch p;
    memset(&p, 0, sizeof p);
    p.st.schip = schip;
    p.wrappers = wrappers;
    p.ipw = ipw;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_fn(p, block), block, step_fn_smem(p, block));
  }
  return sms * per_sm;
}

}  // namespace octax
