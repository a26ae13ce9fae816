/*
 * Octax CHIP-8 environment oracle (see octax_oracle.h for scope and sources).
 *
 * TEST INFRASTRUCTURE ONLY: plain, slow, obviously-correct C. One instance is a
 * struct with a byte per pixel and a full 4 KB RAM; instructions are decoded
 * with a switch that mirrors the opcode table; nothing is bit-packed, fused or
 * reordered. Quirk bits change single opcodes (see QUIRK_* below); with
 * quirks == 0 the classic semantics apply.
 */
#include "octax_oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define QUIRK_SHIFT_USES_VY 0x01u   /* 8XY6/8XYE shift VY (not VX) into VX  */
#define QUIRK_LOADSTORE_INC_I 0x02u /* FX55/FX65 leave I = I + X + 1        */
#define QUIRK_LOGIC_RESETS_VF 0x04u /* 8XY1/8XY2/8XY3 set VF = 0            */
#define QUIRK_JUMP_VX 0x08u         /* BXNN jumps to XNN + VX (not NNN + V0) */
#define QUIRK_WRAP_SPRITES 0x10u    /* DXYN pixels wrap around the edges    */
#define QUIRK_FX1E_VF 0x20u         /* FX1E sets VF = (I + VX > 0xFFF)      */
#define QUIRK_ALL 0x3Fu

/* The conventional 4x5 hexadecimal glyphs, 5 bytes each, stored at 0x050
 * (App. B "Font System" fixes the location 0x050-0x09F; the paper does not
 * print the glyph bytes, so these are the widely used CHIP-8 shapes). */
static const uint8_t ORC_FONT[80] = {
    0xF0, 0x90, 0x90, 0x90, 0xF0, /* 0 */
    0x20, 0x60, 0x20, 0x20, 0x70, /* 1 */
    0xF0, 0x10, 0xF0, 0x80, 0xF0, /* 2 */
    0xF0, 0x10, 0xF0, 0x10, 0xF0, /* 3 */
    0x90, 0x90, 0xF0, 0x10, 0x10, /* 4 */
    0xF0, 0x80, 0xF0, 0x10, 0xF0, /* 5 */
    0xF0, 0x80, 0xF0, 0x90, 0xF0, /* 6 */
    0xF0, 0x10, 0x20, 0x40, 0x40, /* 7 */
    0xF0, 0x90, 0xF0, 0x90, 0xF0, /* 8 */
    0xF0, 0x90, 0xF0, 0x10, 0xF0, /* 9 */
    0xF0, 0x90, 0xF0, 0x90, 0x90, /* A */
    0xE0, 0x90, 0xE0, 0x90, 0xE0, /* B */
    0xF0, 0x80, 0x80, 0x80, 0xF0, /* C */
    0xE0, 0x90, 0x90, 0x90, 0xE0, /* D */
    0xF0, 0x80, 0xF0, 0x80, 0xF0, /* E */
    0xF0, 0x80, 0xF0, 0x80, 0x80  /* F */
};

/* SCHIP 8x10 glyphs at 0x0A0 (FX30). READING: no source fixes their shapes;
 * each is the 4x5 glyph above with every pixel drawn as a 2x2 block (row r
 * of the big glyph is row r/2 of the small one, each of its 4 pixels
 * doubled). Written into RAM at reset of SCHIP games only. */
#define ORC_BIG_FONT_ADDR 0x0A0u
static uint8_t big_glyph_row(uint32_t digit, uint32_t row) {
  uint32_t small = ORC_FONT[5u * digit + row / 2u] >> 4; /* 4 pixels, MSB leftmost */
  uint8_t out = 0;
  for (uint32_t i = 0; i < 4; i++)
    if ((small >> i) & 1u) out = (uint8_t)(out | (3u << (2u * i)));
  return out;
}

size_t orc_frame_bytes(uint32_t variant) { return variant == ORC_SCHIP ? 64u * 128u : 32u * 64u; }

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with the
 * published multipliers, the key bumped by the published Weyl constants
 * between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; round++) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* FNV-1a, 64-bit: offset basis 14695981039346656037, prime 2^40 + 2^8 + 0xb3. */
uint64_t orc_fnv1a64(const uint8_t *p, size_t n) {
  uint64_t h = 14695981039346656037ull;
  for (size_t i = 0; i < n; i++) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

/* ------------------------------------------------------------------------ */
/* Memory: every address wraps to the 4 KB space (App. B: 4 KB memory). */
static uint8_t mem_read(const orc_inst *m, uint32_t addr) { return m->ram[addr % 4096u]; }
static void mem_write(orc_inst *m, uint32_t addr, uint8_t v) { m->ram[addr % 4096u] = v; }

/* Random byte for CXNN. READING: the paper says RND makes games stochastic
 * (§3.2) but not how numbers are drawn; here each draw is one Philox4x32-10
 * block keyed by the seed, counter = (instance uid, env step index,
 * pc | draw index << 16, phase), and the byte is the low 8 bits of word 0. */
static uint8_t random_byte(orc_inst *m, uint32_t pc_of_instr) {
  uint32_t ctr[4], out[4];
  ctr[0] = m->uid;
  ctr[1] = m->env_steps;
  ctr[2] = (pc_of_instr & 0xFFFu) | ((m->draws & 0xFFFFu) << 16);
  ctr[3] = m->phase;
  m->draws++;
  orc_philox4x32_10(ctr, m->key, out);
  return (uint8_t)(out[0] & 0xFFu);
}

/* DXYN (App. B "Sprite Drawing"): XOR an 8-pixel-wide, N-row sprite read from
 * RAM[I..I+N-1] at (VX mod 64, VY mod 32); VF = 1 if any lit pixel was turned
 * off. READING: pixels past the right/bottom edge are clipped (wrapped with
 * QUIRK_WRAP_SPRITES). */
static void draw_sprite(orc_inst *m, uint32_t x, uint32_t y, uint32_t n, uint32_t quirks) {
  uint32_t x0 = m->V[x] % 64u;
  uint32_t y0 = m->V[y] % 32u;
  uint8_t collision = 0;
  for (uint32_t row = 0; row < n; row++) {
    uint8_t bits = mem_read(m, (uint32_t)m->I + row);
    uint32_t py = y0 + row;
    if (py >= 32u) {
      if (quirks & QUIRK_WRAP_SPRITES)
        py %= 32u;
      else
        continue;
    }
    for (uint32_t col = 0; col < 8; col++) {
      uint32_t sprite_pixel = (bits >> (7u - col)) & 1u; /* MSB is leftmost */
      uint32_t px = x0 + col;
      if (px >= 64u) {
        if (quirks & QUIRK_WRAP_SPRITES)
          px %= 64u;
        else
          continue;
      }
      if (sprite_pixel) {
        if (m->pix[py][px]) collision = 1;
        m->pix[py][px] ^= 1u;
      }
    }
  }
  m->V[15] = collision;
}

/* SCHIP DXYN / DXY0 (Super-CHIP 1.1). The screen is a 128x64 buffer. In
 * hires mode sprites use its pixels; in lores mode coordinates are on a 64x32
 * grid and every lit sprite pixel toggles a 2x2 block of the buffer. N = 0
 * draws a 16x16 sprite from 32 bytes at I (two bytes per row, MSB leftmost);
 * READING: 16x16 in both modes. VF = 1 if any toggled buffer pixel was lit
 * (READING: a flag, not the per-row count of the HP48 interpreter). Clipping
 * and the wrap quirk as in CHIP-8, on the grid of the current mode. */
static void draw_sprite_schip(orc_inst *m, uint32_t x, uint32_t y, uint32_t n, uint32_t quirks) {
  uint32_t W = m->hires ? 128u : 64u, H = m->hires ? 64u : 32u;
  uint32_t x0 = m->V[x] % W, y0 = m->V[y] % H;
  uint32_t rows = n == 0 ? 16u : n, cols = n == 0 ? 16u : 8u;
  uint8_t collision = 0;
  for (uint32_t row = 0; row < rows; row++) {
    uint32_t bits = n == 0 ? ((uint32_t)mem_read(m, (uint32_t)m->I + 2u * row) << 8) |
                                 mem_read(m, (uint32_t)m->I + 2u * row + 1u)
                           : mem_read(m, (uint32_t)m->I + row);
    uint32_t py = y0 + row;
    if (py >= H) {
      if (quirks & QUIRK_WRAP_SPRITES)
        py %= H;
      else
        continue;
    }
    for (uint32_t col = 0; col < cols; col++) {
      if (!((bits >> (cols - 1u - col)) & 1u)) continue;
      uint32_t px = x0 + col;
      if (px >= W) {
        if (quirks & QUIRK_WRAP_SPRITES)
          px %= W;
        else
          continue;
      }
      uint32_t s = m->hires ? 1u : 2u; /* buffer pixels per grid pixel */
      for (uint32_t dy = 0; dy < s; dy++)
        for (uint32_t dx = 0; dx < s; dx++) {
          uint8_t *p = &m->pix[py * s + dy][px * s + dx];
          if (*p) collision = 1;
          *p ^= 1u;
        }
    }
  }
  m->V[15] = collision;
}

/* SCHIP scrolls of the 128x64 buffer; vacated pixels are cleared. READING:
 * distances count pixels of the current mode (doubled in lores). */
static void scroll_down(orc_inst *m, uint32_t rows) {
  for (int y = 63; y >= 0; y--)
    for (int x = 0; x < 128; x++) m->pix[y][x] = (uint32_t)y >= rows ? m->pix[y - (int)rows][x] : 0;
}
static void scroll_right(orc_inst *m, uint32_t cols) {
  for (int y = 0; y < 64; y++)
    for (int x = 127; x >= 0; x--) m->pix[y][x] = (uint32_t)x >= cols ? m->pix[y][x - (int)cols] : 0;
}
static void scroll_left(orc_inst *m, uint32_t cols) {
  for (int y = 0; y < 64; y++)
    for (int x = 0; x < 128; x++) m->pix[y][x] = (uint32_t)x + cols < 128u ? m->pix[y][x + (int)cols] : 0;
}

static void set_status(orc_inst *m, uint8_t bit) { m->status |= bit; }

/* One fetch/decode/execute cycle (§3.2 "Fetch-decode-execute cycle"; App. B
 * "Instruction Set Highlights"). key_held is the CHIP-8 key held during this
 * step, or -1. READING: flag-setting ALU ops write VF after VX, so with X = F
 * the flag wins; 8XY5/8XY7 set VF = NOT borrow = (minuend >= subtrahend). */
void orc_exec_one(orc_inst *m, uint32_t quirks, int key_held) {
  uint32_t pc = m->PC;
  uint16_t op = (uint16_t)((mem_read(m, pc) << 8) | mem_read(m, pc + 1u));
  m->PC = (uint16_t)((pc + 2u) % 4096u);

  uint32_t x = (op >> 8) & 0xFu;
  uint32_t y = (op >> 4) & 0xFu;
  uint32_t n = op & 0xFu;
  uint32_t nn = op & 0xFFu;
  uint32_t nnn = op & 0xFFFu;

  const int schip = m->variant == ORC_SCHIP;
  const uint32_t unit = m->hires ? 1u : 2u; /* SCHIP buffer pixels per grid pixel */

  switch (op >> 12) {
    case 0x0:
      if (op == 0x00E0) { /* CLS */
        memset(m->pix, 0, sizeof m->pix);
      } else if (schip && (op & 0xFFF0u) == 0x00C0u) { /* SCHIP 00CN: scroll down N */
        scroll_down(m, n * unit);
      } else if (schip && op == 0x00FB) { /* scroll right 4 */
        scroll_right(m, 4u * unit);
      } else if (schip && op == 0x00FC) { /* scroll left 4 */
        scroll_left(m, 4u * unit);
      } else if (schip && op == 0x00FD) { /* exit. READING: the program stops
                                             here (re-executes) and EXIT is set */
        set_status(m, ORC_ST_EXIT);
        m->PC = (uint16_t)pc;
      } else if (schip && op == 0x00FE) { /* lores. READING: no clear */
        m->hires = 0;
      } else if (schip && op == 0x00FF) { /* hires. READING: no clear */
        m->hires = 1;
      } else if (op == 0x00EE) { /* RET. READING: popping an empty stack faults
                                    and wraps to the top entry. */
        if (m->SP == 0) {
          set_status(m, ORC_ST_STACK_FAULT);
          m->SP = 16;
        }
        m->SP--;
        m->PC = m->stack[m->SP];
      } /* other 0NNN: machine-code call, ignored */
      break;
    case 0x1: /* JP NNN */
      m->PC = (uint16_t)nnn;
      break;
    case 0x2: /* CALL NNN. READING: pushing onto a full 16-entry stack faults
                 and wraps to entry 0. */
      if (m->SP == 16) {
        set_status(m, ORC_ST_STACK_FAULT);
        m->SP = 0;
      }
      m->stack[m->SP] = m->PC;
      m->SP++;
      m->PC = (uint16_t)nnn;
      break;
    case 0x3: /* SE VX, NN */
      if (m->V[x] == nn) m->PC = (uint16_t)((m->PC + 2u) % 4096u);
      break;
    case 0x4: /* SNE VX, NN */
      if (m->V[x] != nn) m->PC = (uint16_t)((m->PC + 2u) % 4096u);
      break;
    case 0x5: /* SE VX, VY */
      if (n != 0) {
        set_status(m, ORC_ST_BAD_OP);
        break;
      }
      if (m->V[x] == m->V[y]) m->PC = (uint16_t)((m->PC + 2u) % 4096u);
      break;
    case 0x6: /* LD VX, NN */
      m->V[x] = (uint8_t)nn;
      break;
    case 0x7: /* ADD VX, NN (no flag) */
      m->V[x] = (uint8_t)((m->V[x] + nn) % 256u);
      break;
    case 0x8: {
      uint32_t vx = m->V[x], vy = m->V[y];
      switch (n) {
        case 0x0:
          m->V[x] = (uint8_t)vy;
          break;
        case 0x1:
          m->V[x] = (uint8_t)(vx | vy);
          if (quirks & QUIRK_LOGIC_RESETS_VF) m->V[15] = 0;
          break;
        case 0x2:
          m->V[x] = (uint8_t)(vx & vy);
          if (quirks & QUIRK_LOGIC_RESETS_VF) m->V[15] = 0;
          break;
        case 0x3:
          m->V[x] = (uint8_t)(vx ^ vy);
          if (quirks & QUIRK_LOGIC_RESETS_VF) m->V[15] = 0;
          break;
        case 0x4: { /* ADD with carry */
          uint32_t sum = vx + vy;
          m->V[x] = (uint8_t)(sum % 256u);
          m->V[15] = (uint8_t)(sum > 255u ? 1 : 0);
          break;
        }
        case 0x5: { /* SUB, VF = NOT borrow */
          uint8_t not_borrow = (uint8_t)(vx >= vy ? 1 : 0);
          m->V[x] = (uint8_t)((vx + 256u - vy) % 256u);
          m->V[15] = not_borrow;
          break;
        }
        case 0x6: { /* SHR, VF = bit shifted out */
          uint32_t src = (quirks & QUIRK_SHIFT_USES_VY) ? vy : vx;
          uint8_t out_bit = (uint8_t)(src & 1u);
          m->V[x] = (uint8_t)(src / 2u);
          m->V[15] = out_bit;
          break;
        }
        case 0x7: { /* SUBN: VX = VY - VX, VF = NOT borrow */
          uint8_t not_borrow = (uint8_t)(vy >= vx ? 1 : 0);
          m->V[x] = (uint8_t)((vy + 256u - vx) % 256u);
          m->V[15] = not_borrow;
          break;
        }
        case 0xE: { /* SHL, VF = bit shifted out */
          uint32_t src = (quirks & QUIRK_SHIFT_USES_VY) ? vy : vx;
          uint8_t out_bit = (uint8_t)((src >> 7) & 1u);
          m->V[x] = (uint8_t)((src * 2u) % 256u);
          m->V[15] = out_bit;
          break;
        }
        default:
          set_status(m, ORC_ST_BAD_OP);
          break;
      }
      break;
    }
    case 0x9: /* SNE VX, VY */
      if (n != 0) {
        set_status(m, ORC_ST_BAD_OP);
        break;
      }
      if (m->V[x] != m->V[y]) m->PC = (uint16_t)((m->PC + 2u) % 4096u);
      break;
    case 0xA: /* LD I, NNN */
      m->I = (uint16_t)nnn;
      break;
    case 0xB: /* JP V0, NNN */
      if (quirks & QUIRK_JUMP_VX)
        m->PC = (uint16_t)((nnn + m->V[x]) % 4096u);
      else
        m->PC = (uint16_t)((nnn + m->V[0]) % 4096u);
      break;
    case 0xC: /* RND VX, NN */
      m->V[x] = (uint8_t)(random_byte(m, pc) & nn);
      break;
    case 0xD: /* DRW VX, VY, N */
      if (schip)
        draw_sprite_schip(m, x, y, n, quirks);
      else
        draw_sprite(m, x, y, n, quirks);
      break;
    case 0xE: {
      int pressed = (key_held >= 0) && ((uint32_t)key_held == (m->V[x] & 0xFu));
      if (nn == 0x9E) { /* SKP VX */
        if (pressed) m->PC = (uint16_t)((m->PC + 2u) % 4096u);
      } else if (nn == 0xA1) { /* SKNP VX */
        if (!pressed) m->PC = (uint16_t)((m->PC + 2u) % 4096u);
      } else {
        set_status(m, ORC_ST_BAD_OP);
      }
      break;
    }
    case 0xF:
      switch (nn) {
        case 0x07:
          m->V[x] = m->DT;
          break;
        case 0x0A: /* LD VX, K. READING: proceeds when a key is held (the
                      step's key), otherwise re-executes; no release wait. */
          if (key_held >= 0)
            m->V[x] = (uint8_t)key_held;
          else
            m->PC = (uint16_t)((m->PC + 4096u - 2u) % 4096u);
          break;
        case 0x15:
          m->DT = m->V[x];
          break;
        case 0x18:
          m->ST = m->V[x];
          break;
        case 0x1E: {
          uint32_t sum = (uint32_t)m->I + m->V[x];
          if (quirks & QUIRK_FX1E_VF) {
            m->I = (uint16_t)(sum % 65536u);
            m->V[15] = (uint8_t)(sum > 0xFFFu ? 1 : 0);
          } else {
            m->I = (uint16_t)(sum % 65536u);
          }
          break;
        }
        case 0x29: /* LD F, VX: glyph of the low digit of VX */
          m->I = (uint16_t)(0x50u + 5u * (m->V[x] % 16u));
          break;
        case 0x30: /* SCHIP LD HF, VX: 8x10 glyph of the low digit of VX */
          if (!schip) {
            set_status(m, ORC_ST_BAD_OP);
            break;
          }
          m->I = (uint16_t)(ORC_BIG_FONT_ADDR + 10u * (m->V[x] % 16u));
          break;
        case 0x75: /* SCHIP: flags[0..X] = V0..VX. READING: 16 flag bytes */
          if (!schip) {
            set_status(m, ORC_ST_BAD_OP);
            break;
          }
          for (uint32_t i = 0; i <= x; i++) m->rpl[i] = m->V[i];
          break;
        case 0x85: /* SCHIP: V0..VX = flags[0..X] */
          if (!schip) {
            set_status(m, ORC_ST_BAD_OP);
            break;
          }
          for (uint32_t i = 0; i <= x; i++) m->V[i] = m->rpl[i];
          break;
        case 0x33: { /* BCD */
          uint32_t v = m->V[x];
          mem_write(m, (uint32_t)m->I + 0u, (uint8_t)(v / 100u));
          mem_write(m, (uint32_t)m->I + 1u, (uint8_t)((v / 10u) % 10u));
          mem_write(m, (uint32_t)m->I + 2u, (uint8_t)(v % 10u));
          break;
        }
        case 0x55: /* store V0..VX at I. READING (fixed quirk set): I unchanged */
          for (uint32_t i = 0; i <= x; i++) mem_write(m, (uint32_t)m->I + i, m->V[i]);
          if (quirks & QUIRK_LOADSTORE_INC_I) m->I = (uint16_t)((m->I + x + 1u) % 65536u);
          break;
        case 0x65: /* load V0..VX from I */
          for (uint32_t i = 0; i <= x; i++) m->V[i] = mem_read(m, (uint32_t)m->I + i);
          if (quirks & QUIRK_LOADSTORE_INC_I) m->I = (uint16_t)((m->I + x + 1u) % 65536u);
          break;
        default:
          set_status(m, ORC_ST_BAD_OP);
          break;
      }
      break;
  }
}

/* 60 Hz timers (App. B "Timers"; §3.2): one tick per emulated frame. */
void orc_tick_timers(orc_inst *m) {
  if (m->DT > 0) m->DT--;
  if (m->ST > 0) m->ST--;
}

/* ------------------------------------------------------------------------ */
/* score_fn / terminated_fn (§3.3 "Score function design", "Termination
 * logic"; App. C game list). */
static int32_t term_value(const orc_inst *m, const orc_term *t) {
  int32_t v;
  if (t->src == ORC_SRC_REG)
    v = m->V[t->idx & 15];
  else
    v = m->ram[t->idx & 0xFFF];
  switch (t->xform) {
    case ORC_X_RAW: return v;
    case ORC_X_NEG: return -v;
    case ORC_X_DEC_TENS: return v / 10;
    case ORC_X_DEC_ONES: return v % 10;
    case ORC_X_DEC_TENS_MINUS_ONES: return v / 10 - v % 10;
    case ORC_X_NIB_HI_MINUS_LO: return (v / 16) - (v % 16);
    case ORC_X_ZERO_IF_GT: return v > t->arg ? 0 : v;
    default: return 0;
  }
}

int32_t orc_score(const orc_inst *m, const orc_game *g) {
  int32_t s = 0;
  for (uint32_t i = 0; i < g->n_score_terms; i++) s += term_value(m, &g->score[i]);
  return s;
}

int orc_terminated(const orc_inst *m, const orc_game *g) {
  for (uint32_t i = 0; i < g->n_term_clauses; i++) {
    const orc_clause *c = &g->term[i];
    int32_t v = term_value(m, &c->lhs);
    int hit = 0;
    switch (c->cmp) {
      case ORC_EQ: hit = v == c->rhs; break;
      case ORC_NE: hit = v != c->rhs; break;
      case ORC_GE: hit = v >= c->rhs; break;
      case ORC_GT: hit = v > c->rhs; break;
      case ORC_LE: hit = v <= c->rhs; break;
      case ORC_LT: hit = v < c->rhs; break;
    }
    if (hit) return 1;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* A 32-bit draw for the environment wrappers (READING: Philox4x32-10, word
 * 0, counter = (uid, env step index, 0, phase) with phase 2 for the sticky
 * action test and 3 for the no-op count; phases 0/1 belong to CXNN). */
static uint32_t wrapper_draw(const orc_inst *m, uint32_t phase) {
  uint32_t ctr[4] = {m->uid, m->env_steps, 0u, phase}, out[4];
  orc_philox4x32_10(ctr, m->key, out);
  return out[0];
}

/* Reset (§3.2 "ROM loading and initialization", "Environment integration";
 * §3.3 "Initialization handling"): RAM cleared, font at 0x050, ROM at 0x200,
 * registers, timers, stack and display cleared, PC = 0x200, then the game's
 * startup instructions run with no key held. READING: timers tick after every
 * K startup instructions, as in normal frames. The env step counter, the
 * random identity and the sticky status bits are kept.
 * No-op reset (§3.2, "wrappers for no-op reset"): READING: after the startup
 * instructions, a drawn number of no-key env steps (frameskip frames of K
 * instructions and a timer tick each, nothing observed) in 0..max_noops. */
int orc_inst_reset(orc_inst *m, const orc_game *g, uint32_t quirks) {
  if (g->rom_len > 4096u - 0x200u) return -1;
  memset(m->V, 0, sizeof m->V);
  m->I = 0;
  m->PC = 0x200;
  m->SP = 0;
  m->DT = 0;
  m->ST = 0;
  memset(m->stack, 0, sizeof m->stack);
  memset(m->pix, 0, sizeof m->pix);
  memset(m->ram, 0, sizeof m->ram);
  memcpy(m->ram + 0x50, ORC_FONT, sizeof ORC_FONT);
  m->variant = (uint8_t)g->variant;
  m->hires = 0;                       /* READING: every episode starts in lores */
  memset(m->rpl, 0, sizeof m->rpl);   /* READING: flags do not outlive an episode */
  if (g->variant == ORC_SCHIP)
    for (uint32_t d = 0; d < 16; d++)
      for (uint32_t r = 0; r < 10; r++) m->ram[ORC_BIG_FONT_ADDR + 10u * d + r] = big_glyph_row(d, r);
  memcpy(m->ram + 0x200, g->rom, g->rom_len);
  m->episode_steps = 0;
  m->phase = 1;
  m->draws = 0;
  for (uint32_t i = 0; i < g->startup_instrs; i++) {
    orc_exec_one(m, quirks, -1);
    if ((i + 1) % g->instr_per_frame == 0) orc_tick_timers(m);
  }
  if (g->max_noops > 0) {
    uint32_t noops = wrapper_draw(m, 3) % (g->max_noops + 1u);
    for (uint32_t s = 0; s < noops; s++)
      for (uint32_t f = 0; f < g->frameskip; f++) {
        for (uint32_t k = 0; k < g->instr_per_frame; k++) orc_exec_one(m, quirks, -1);
        orc_tick_timers(m);
      }
  }
  m->last_action = (uint8_t)g->n_actions;  /* the previous action of a new episode: no-op */
  m->phase = 0;
  m->draws = 0;
  return 0;
}

/* One observation frame: the 64x32 screen (CHIP-8) or the 128x64 buffer (SCHIP). */
static void write_frame(const orc_inst *m, uint8_t *dst) {
  int W = m->variant == ORC_SCHIP ? 128 : 64, H = m->variant == ORC_SCHIP ? 64 : 32;
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++) dst[y * W + x] = m->pix[y][x];
}

/* One environment step (§3.2 "Environment integration", §4.2): the action's
 * key is held for the whole step; frameskip frames of K instructions, each
 * followed by a timer tick and a frame capture; the observation is the last
 * stack_frames frames, oldest first (READING: frames at frame granularity).
 * reward = score after - score before (READING: the returns reported in §4.3
 * equal final scores, so reward is the score increase). done = terminated or
 * truncated; a done instance is reset and its observation is the reset display
 * repeated (READING: auto-reset, terminal reward/done, reset observation). */
int orc_inst_step(orc_inst *m, const orc_game *g, uint32_t quirks, uint32_t action,
                  uint8_t *obs, float *reward, uint8_t *done) {
  /* Sticky actions (§3.2, "wrappers for ... sticky actions"). READING: per
   * env step, with probability sticky_threshold / 2^32 the previous step's
   * action is applied instead of the agent's. */
  if (g->sticky_threshold > 0 && wrapper_draw(m, 2) < g->sticky_threshold) action = m->last_action;
  m->last_action = (uint8_t)(action > 255u ? 255u : action);
  int key = -1;
  if (action < g->n_actions)
    key = g->action_set[action] & 15;
  else if (action > g->n_actions)
    set_status(m, ORC_ST_BAD_ACTION); /* out-of-range index acts as no-op */

  int32_t score_before = orc_score(m, g);
  m->phase = 0;
  m->draws = 0;
  for (uint32_t f = 0; f < g->frameskip; f++) {
    for (uint32_t k = 0; k < g->instr_per_frame; k++) orc_exec_one(m, quirks, key);
    orc_tick_timers(m);
    uint32_t first_kept = g->frameskip - g->stack_frames;
    if (obs && f >= first_kept) write_frame(m, obs + (size_t)(f - first_kept) * orc_frame_bytes(g->variant));
  }
  int32_t score_after = orc_score(m, g);
  m->episode_steps++;
  m->env_steps++;
  int term = orc_terminated(m, g);
  int trunc = g->max_episode_steps > 0 && m->episode_steps >= g->max_episode_steps;
  *reward = (float)(score_after - score_before);
  *done = (uint8_t)((term || trunc) ? 1 : 0);
  if (*done) {
    orc_inst_reset(m, g, quirks);
    if (obs)
      for (uint32_t s = 0; s < g->stack_frames; s++) write_frame(m, obs + (size_t)s * orc_frame_bytes(g->variant));
  }
  return 0;
}

void orc_inst_record(const orc_inst *m, orc_record *r) {
  memset(r, 0, sizeof *r);
  memcpy(r->V, m->V, 16);
  r->I = m->I;
  r->PC = m->PC;
  r->SP = m->SP;
  r->DT = m->DT;
  r->ST = m->ST;
  r->status = m->status;
  memcpy(r->stack, m->stack, sizeof r->stack);
  for (int y = 0; y < 64; y++)
    for (int h = 0; h < 2; h++) {
      uint64_t w = 0;
      for (int x = 0; x < 64; x++)
        if (m->pix[y][64 * h + x]) w |= (uint64_t)1 << x;
      r->display[y][h] = w;
    }
  memcpy(r->ram, m->ram, 4096);
  r->episode_steps = m->episode_steps;
  r->env_steps = m->env_steps;
  r->last_action = m->last_action;
  r->hires = m->hires;
  memcpy(r->rpl, m->rpl, 16);
}

/* Serialise the record field by field, little-endian, then FNV-1a. CHIP-8:
 * the display is rows 0-31, word 0. SCHIP: all 64 x 2 words (row-major),
 * followed after last_action by hires and the 16 flag bytes. */
uint64_t orc_inst_hash(const orc_inst *m) {
  orc_record r;
  orc_inst_record(m, &r);
  const int schip = m->variant == ORC_SCHIP;
  uint8_t buf[5300];
  size_t o = 0;
  memcpy(buf + o, r.V, 16); o += 16;
  buf[o++] = (uint8_t)(r.I & 0xFF); buf[o++] = (uint8_t)(r.I >> 8);
  buf[o++] = (uint8_t)(r.PC & 0xFF); buf[o++] = (uint8_t)(r.PC >> 8);
  buf[o++] = r.SP; buf[o++] = r.DT; buf[o++] = r.ST; buf[o++] = r.status;
  for (int i = 0; i < 16; i++) {
    buf[o++] = (uint8_t)(r.stack[i] & 0xFF);
    buf[o++] = (uint8_t)(r.stack[i] >> 8);
  }
  for (int y = 0; y < (schip ? 64 : 32); y++)
    for (int h = 0; h < (schip ? 2 : 1); h++)
      for (int b = 0; b < 8; b++) buf[o++] = (uint8_t)(r.display[y][h] >> (8 * b));
  memcpy(buf + o, r.ram, 4096); o += 4096;
  for (int b = 0; b < 4; b++) buf[o++] = (uint8_t)(r.episode_steps >> (8 * b));
  for (int b = 0; b < 4; b++) buf[o++] = (uint8_t)(r.env_steps >> (8 * b));
  buf[o++] = r.last_action;
  if (schip) {
    buf[o++] = r.hires;
    memcpy(buf + o, r.rpl, 16); o += 16;
  }
  return orc_fnv1a64(buf, o);
}

/* ------------------------------------------------------------------------ */
/* The batch: a plain loop over independent instances (the paper's vmap over
 * environments, §3.2 / §4.2). Threads split the instance range; they never
 * interact. */
struct orc_env {
  orc_game *games;
  uint8_t **roms;
  int n_games;
  int64_t n;
  uint32_t quirks;
  orc_inst *inst;
  int stack_frames;
};

orc_env *orc_env_create(const orc_game *games, int n_games, const uint16_t *game_of_env,
                        const uint32_t *uid_of_env, int64_t n_envs, uint32_t quirks,
                        uint64_t seed) {
  if (n_games <= 0 || n_envs < 0 || (quirks & ~QUIRK_ALL)) return NULL;
  for (int gi = 0; gi < n_games; gi++) {
    const orc_game *g = &games[gi];
    if (g->rom_len == 0 || g->rom_len > 3584u || g->instr_per_frame == 0 || g->frameskip == 0 ||
        g->stack_frames == 0 || g->stack_frames > g->frameskip || g->n_actions > 16 ||
        g->n_score_terms > 4 || g->n_term_clauses > 4 || g->variant > ORC_SCHIP ||
        g->stack_frames != games[0].stack_frames || g->variant != games[0].variant)
      return NULL;
  }
  orc_env *e = (orc_env *)calloc(1, sizeof *e);
  e->n_games = n_games;
  e->n = n_envs;
  e->quirks = quirks;
  e->stack_frames = (int)games[0].stack_frames;
  e->games = (orc_game *)calloc((size_t)n_games, sizeof(orc_game));
  e->roms = (uint8_t **)calloc((size_t)n_games, sizeof(uint8_t *));
  for (int gi = 0; gi < n_games; gi++) {
    e->games[gi] = games[gi];
    e->roms[gi] = (uint8_t *)malloc(games[gi].rom_len);
    memcpy(e->roms[gi], games[gi].rom, games[gi].rom_len);
    e->games[gi].rom = e->roms[gi];
  }
  e->inst = (orc_inst *)calloc((size_t)(n_envs > 0 ? n_envs : 1), sizeof(orc_inst));
  for (int64_t i = 0; i < n_envs; i++) {
    orc_inst *m = &e->inst[i];
    int gi = game_of_env ? game_of_env[i] : 0;
    if (gi >= n_games) {
      orc_env_destroy(e);
      return NULL;
    }
    m->game = gi;
    m->uid = uid_of_env ? uid_of_env[i] : (uint32_t)i;
    m->key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
    m->key[1] = (uint32_t)(seed >> 32);
    m->env_steps = 0;
    m->status = 0;
    orc_inst_reset(m, &e->games[gi], quirks);
  }
  return e;
}

int orc_env_reset(orc_env *e, const uint8_t *mask, uint8_t *obs) {
  const size_t fb = orc_frame_bytes(e->games[0].variant);
  size_t per = (size_t)e->stack_frames * fb;
  for (int64_t i = 0; i < e->n; i++) {
    if (mask && !mask[i]) continue;
    orc_inst *m = &e->inst[i];
    orc_inst_reset(m, &e->games[m->game], e->quirks);
    if (obs)
      for (int s = 0; s < e->stack_frames; s++) write_frame(m, obs + per * (size_t)i + (size_t)s * fb);
  }
  return 0;
}

typedef struct {
  orc_env *e;
  int64_t lo, hi;
  const uint8_t *actions;
  uint8_t *obs;
  float *reward;
  uint8_t *done;
} step_job;

static void *step_range(void *arg) {
  step_job *j = (step_job *)arg;
  orc_env *e = j->e;
  size_t per = (size_t)e->stack_frames * orc_frame_bytes(e->games[0].variant);
  for (int64_t i = j->lo; i < j->hi; i++) {
    orc_inst *m = &e->inst[i];
    float r;
    uint8_t d;
    orc_inst_step(m, &e->games[m->game], e->quirks, j->actions[i], j->obs ? j->obs + per * (size_t)i : NULL, &r, &d);
    if (j->reward) j->reward[i] = r;
    if (j->done) j->done[i] = d;
  }
  return NULL;
}

int orc_env_step(orc_env *e, const uint8_t *actions, uint8_t *obs, float *reward, uint8_t *done,
                 int n_threads) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  if ((int64_t)n_threads > e->n) n_threads = e->n > 0 ? (int)e->n : 1;
  step_job jobs[256];
  pthread_t tids[256];
  for (int t = 0; t < n_threads; t++) {
    jobs[t].e = e;
    jobs[t].lo = e->n * t / n_threads;
    jobs[t].hi = e->n * (t + 1) / n_threads;
    jobs[t].actions = actions;
    jobs[t].obs = obs;
    jobs[t].reward = reward;
    jobs[t].done = done;
  }
  if (n_threads == 1) {
    step_range(&jobs[0]);
    return 0;
  }
  for (int t = 0; t < n_threads; t++) pthread_create(&tids[t], NULL, step_range, &jobs[t]);
  for (int t = 0; t < n_threads; t++) pthread_join(tids[t], NULL);
  return 0;
}

int orc_env_hash(const orc_env *e, uint64_t *out) {
  for (int64_t i = 0; i < e->n; i++) out[i] = orc_inst_hash(&e->inst[i]);
  return 0;
}

int orc_env_records(const orc_env *e, orc_record *out) {
  for (int64_t i = 0; i < e->n; i++) orc_inst_record(&e->inst[i], &out[i]);
  return 0;
}

orc_inst *orc_env_inst(orc_env *e, int64_t i) { return (i >= 0 && i < e->n) ? &e->inst[i] : NULL; }
int64_t orc_env_size(const orc_env *e) { return e->n; }

void orc_env_destroy(orc_env *e) {
  if (!e) return;
  for (int gi = 0; gi < e->n_games; gi++) free(e->roms[gi]);
  free(e->roms);
  free(e->games);
  free(e->inst);
  free(e);
}

int orc_env_rollout(orc_env *e, int n_steps, const uint8_t *actions, uint8_t *obs, float *reward,
                    uint8_t *done, uint64_t *hashes, int n_threads) {
  size_t per = (size_t)e->stack_frames * orc_frame_bytes(e->games[0].variant);
  for (int s = 0; s < n_steps; s++) {
    orc_env_step(e, actions + (size_t)s * (size_t)e->n, obs ? obs + (size_t)s * (size_t)e->n * per : NULL,
                 reward ? reward + (size_t)s * (size_t)e->n : NULL, done ? done + (size_t)s * (size_t)e->n : NULL,
                 n_threads);
    if (hashes) orc_env_hash(e, hashes + (size_t)s * (size_t)e->n);
  }
  return 0;
}
