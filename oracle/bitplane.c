/*
 * Oracle: exponent alignment, Algorithm 1 (bitplane encoding) and its
 * inverse.  TEST INFRASTRUCTURE ONLY (see hpmdr_oracle.h).
 *
 * Algorithm 1 (Sec. 4) aligns the decomposed array to its maximum exponent and
 * then, for b = B-1 down to 0, stores bit b of every aligned element as one
 * bitplane.  Readings used where the paper is silent:
 *   - alignment per level: bl = bit length of max|C8| over the level and
 *     q = |C8| << (B - bl) if B >= bl, else |C8| >> (bl - B) (floor), so q < 2^B;
 *   - sign-magnitude: one extra sign plane (bit = C8 < 0) stored first;
 *   - element j of the level goes to word j >> 5, bit j & 31 of each plane;
 *     every plane is padded with zero bits to 4*ceil(n/128) words;
 *   - stream plane p = 0 is magnitude bit B-1 (the loop order of Alg. 1);
 *   - merged groups of m = 4 planes (Sec. 5.2): group 0 = sign + p0..p3,
 *     group g >= 1 = p4g..p4g+3.
 */
#include <string.h>

#include "hpmdr_oracle.h"

static int bitlen_u64(uint64_t v) {
  int b = 0;
  while (v) {
    b++;
    v >>= 1;
  }
  return b;
}

static uint64_t magnitude(int64_t c) { return c < 0 ? (uint64_t)(-c) : (uint64_t)c; }

int or_bitlen_max(const int64_t* C8, uint64_t n) {
  uint64_t m = 0;
  for (uint64_t j = 0; j < n; j++)
    if (magnitude(C8[j]) > m) m = magnitude(C8[j]);
  return bitlen_u64(m);
}

/* AlignExponent of Alg. 1, applied per level */
void or_quantize(const int64_t* C8, uint64_t n, int B, int bl, uint64_t* q, uint8_t* sign) {
  for (uint64_t j = 0; j < n; j++) {
    uint64_t a = magnitude(C8[j]);
    if (bl == 0) q[j] = 0;
    else if (B >= bl) q[j] = a << (B - bl);
    else q[j] = a >> (bl - B);
    sign[j] = (uint8_t)(C8[j] < 0);
  }
}

/* 1 when the dropped low bits (bl > B) are zero for every coefficient */
int or_level_exact(const int64_t* C8, uint64_t n, int B, int bl) {
  if (bl <= B) return 1;
  for (uint64_t j = 0; j < n; j++)
    if (magnitude(C8[j]) & ((1ull << (bl - B)) - 1)) return 0;
  return 1;
}

static void set_bit(uint32_t* plane, uint64_t j, unsigned bit) {
  plane[j >> 5] |= (uint32_t)bit << (j & 31);
}

static unsigned get_bit(const uint32_t* plane, uint64_t j) {
  return (plane[j >> 5] >> (j & 31)) & 1u;
}

/* Alg. 1: for b = B-1 .. 0 extract bit b of every element into one plane */
void or_bitplane_encode(const uint64_t* q, const uint8_t* sign, uint64_t n, int B,
                        uint32_t* planes) {
  uint64_t W = or_plane_words(n);
  memset(planes, 0, (size_t)(B + 1) * W * 4);
  for (uint64_t j = 0; j < n; j++) set_bit(planes, j, sign[j] & 1u);
  for (int b = B - 1; b >= 0; b--) {
    int p = B - 1 - b;
    uint32_t* plane = planes + (uint64_t)(1 + p) * W;
    for (uint64_t j = 0; j < n; j++) set_bit(plane, j, (unsigned)((q[j] >> b) & 1u));
  }
}

void or_bitplane_decode(const uint32_t* planes, uint64_t n, int B, int k, uint64_t* q_hat,
                        uint8_t* sign) {
  uint64_t W = or_plane_words(n);
  for (uint64_t j = 0; j < n; j++) {
    uint64_t v = 0;
    for (int p = 0; p < k; p++)
      v |= (uint64_t)get_bit(planes + (uint64_t)(1 + p) * W, j) << (B - 1 - p);
    q_hat[j] = v;
    sign[j] = (uint8_t)(k > 0 ? get_bit(planes, j) : 0);
  }
}

/* coefficient from the fetched bits: truncation, no midpoint */
int64_t or_dequantize(uint64_t qhat, int s, int B, int bl) {
  uint64_t a;
  if (bl == 0) a = 0;
  else if (B >= bl) a = qhat >> (B - bl);
  else a = qhat << (bl - B);
  return s ? -(int64_t)a : (int64_t)a;
}

int or_num_groups(int B) { return B / 4; }

uint64_t or_group_offset(uint64_t W, int g) {
  return g == 0 ? 0 : (uint64_t)(4 * g + 1) * W * 4;
}

uint64_t or_group_size(uint64_t W, int g) { return (uint64_t)(g == 0 ? 5 : 4) * W * 4; }
