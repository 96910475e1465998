/*
 * Oracle: the lossless coders of Sec. 5.1 and the hybrid choice of
 * Algorithm 2 (Sec. 5.2).  TEST INFRASTRUCTURE ONLY (see hpmdr_oracle.h).
 *
 * The paper cites its Huffman and RLE implementations without fixing formats.
 * Readings used:
 *   Huffman: byte symbols; code lengths from the two-queue construction (leaf
 *     queue sorted by (frequency, symbol), a leaf wins a weight tie against an
 *     internal node, internal nodes taken in creation order); lengths capped at
 *     16 by halving the counts (f <- (f+1)>>1 for f>0) and rebuilding; a lone
 *     symbol gets length 1; canonical codes in (length, symbol) order written
 *     MSB-first into 32-bit words; the input is cut into 16 KiB chunks that
 *     each start on a fresh word.  Layout: u64 orig_len, u32 chunk_bytes,
 *     u32 nchunks, u8 len[256], u32 word_off[nchunks+1], payload words.
 *     Ratio estimate (Sec. 5.2, "Huffman compression ratio estimation"):
 *     header + ceil(sum f*len / 8) + 4*nchunks bytes.
 *   RLE: byte runs inside 16 KiB chunks, each run stored as the byte followed
 *     by LEB128(run-1).  Layout: u64 orig_len, u32 chunk_bytes, u32 nchunks,
 *     u32 byte_off[nchunks+1], payload.  The estimate of Sec. 5.2 ("RLE
 *     compression ratio estimation") is the exact encoded size.
 *   DC: the group bytes as they are.
 *   Alg. 2: S > T_s (strict), then Huffman if S/est_H > T_cr, else RLE if
 *     S/est_R > T_cr, else DC; ratios compared exactly as S*den > num*est.
 */
#include <stdlib.h>
#include <string.h>

#include "hpmdr_oracle.h"

typedef unsigned __int128 u128;

static uint64_t nchunks_of(uint64_t S) { return (S + OR_CHUNK_BYTES - 1) / OR_CHUNK_BYTES; }

static void put_u32(uint8_t* p, uint32_t v) { memcpy(p, &v, 4); }
static void put_u64(uint8_t* p, uint64_t v) { memcpy(p, &v, 8); }
static uint32_t get_u32(const uint8_t* p) { uint32_t v; memcpy(&v, p, 4); return v; }
static uint64_t get_u64(const uint8_t* p) { uint64_t v; memcpy(&v, p, 8); return v; }

void or_histogram(const uint8_t* G, uint64_t S, uint64_t hist[256]) {
  memset(hist, 0, 256 * sizeof(uint64_t));
  for (uint64_t i = 0; i < S; i++) hist[G[i]]++;
}

/* ---------------------------------------------------------------- Huffman */

/* one Huffman construction with the two-queue method; returns max length */
static int huffman_build(const uint64_t f[256], uint8_t len[256]) {
  int sym[256], n = 0, maxlen = 0;
  uint64_t w[511];
  int parent[511], depth[511];
  memset(len, 0, 256);
  for (int s = 0; s < 256; s++)
    if (f[s] > 0) sym[n++] = s;
  if (n == 0) return 0;
  if (n == 1) {
    len[sym[0]] = 1;
    return 1;
  }
  /* leaf queue sorted by (frequency, symbol): insertion sort on n <= 256 */
  for (int a = 1; a < n; a++) {
    int s = sym[a], b = a - 1;
    while (b >= 0 && (f[sym[b]] > f[s] || (f[sym[b]] == f[s] && sym[b] > s))) {
      sym[b + 1] = sym[b];
      b--;
    }
    sym[b + 1] = s;
  }
  for (int i = 0; i < n; i++) w[i] = f[sym[i]];
  int next_leaf = 0, next_int = n, created = n;
  for (int step = 0; step < n - 1; step++) {
    int pick[2];
    for (int k = 0; k < 2; k++) {
      int leaf_ok = next_leaf < n, int_ok = next_int < created;
      if (leaf_ok && (!int_ok || w[next_leaf] <= w[next_int])) pick[k] = next_leaf++;
      else pick[k] = next_int++;
    }
    w[created] = w[pick[0]] + w[pick[1]];
    parent[pick[0]] = created;
    parent[pick[1]] = created;
    created++;
  }
  /* node indices grow with creation, so parents come after their children */
  depth[created - 1] = 0;
  for (int v = created - 2; v >= 0; v--) depth[v] = depth[parent[v]] + 1;
  for (int i = 0; i < n; i++) {
    len[sym[i]] = (uint8_t)depth[i];
    if (depth[i] > maxlen) maxlen = depth[i];
  }
  return maxlen;
}

void or_huffman_lengths(const uint64_t hist[256], uint8_t len[256]) {
  uint64_t f[256];
  memcpy(f, hist, sizeof(f));
  while (huffman_build(f, len) > 16)
    for (int s = 0; s < 256; s++)
      if (f[s] > 0) f[s] = (f[s] + 1) >> 1;
}

static uint64_t huffman_header_bytes(uint64_t nchunks) { return 8 + 4 + 4 + 256 + 4 * (nchunks + 1); }

uint64_t or_huffman_estimate(const uint64_t hist[256], const uint8_t len[256], uint64_t S) {
  u128 bits = 0;
  uint64_t nc = nchunks_of(S);
  for (int s = 0; s < 256; s++) bits += (u128)hist[s] * len[s];
  return huffman_header_bytes(nc) + (uint64_t)((bits + 7) / 8) + 4 * nc;
}

/* canonical codes in (length, symbol) order */
static void canonical_codes(const uint8_t len[256], uint32_t code[256]) {
  uint32_t c = 0;
  int prev = 0, first = 1;
  memset(code, 0, 256 * sizeof(uint32_t));
  for (int L = 1; L <= 16; L++)
    for (int s = 0; s < 256; s++) {
      if (len[s] != L) continue;
      if (first) {
        c = 0;
        first = 0;
      } else {
        c = (c + 1) << (L - prev);
      }
      prev = L;
      code[s] = c;
    }
}

uint64_t or_huffman_encode(const uint8_t* G, uint64_t S, uint8_t* out) {
  uint64_t hist[256];
  uint8_t len[256];
  uint32_t code[256];
  uint64_t nc = nchunks_of(S), hdr = huffman_header_bytes(nc), words = 0;
  or_histogram(G, S, hist);
  or_huffman_lengths(hist, len);
  canonical_codes(len, code);
  /* payload words per chunk */
  uint32_t* off = (uint32_t*)malloc((nc + 1) * sizeof(uint32_t));
  for (uint64_t c = 0; c < nc; c++) {
    uint64_t bits = 0, end = (c + 1) * OR_CHUNK_BYTES < S ? (c + 1) * OR_CHUNK_BYTES : S;
    for (uint64_t i = c * OR_CHUNK_BYTES; i < end; i++) bits += len[G[i]];
    off[c] = (uint32_t)words;
    words += (bits + 31) / 32;
  }
  off[nc] = (uint32_t)words;
  if (out) {
    uint32_t* payload = (uint32_t*)calloc(words ? words : 1, sizeof(uint32_t));
    for (uint64_t c = 0; c < nc; c++) {
      uint64_t pos = (uint64_t)off[c] * 32;
      uint64_t end = (c + 1) * OR_CHUNK_BYTES < S ? (c + 1) * OR_CHUNK_BYTES : S;
      for (uint64_t i = c * OR_CHUNK_BYTES; i < end; i++) {
        int L = len[G[i]];
        for (int b = L - 1; b >= 0; b--, pos++) /* MSB of the code first */
          payload[pos >> 5] |= ((code[G[i]] >> b) & 1u) << (31 - (pos & 31));
      }
    }
    put_u64(out, S);
    put_u32(out + 8, OR_CHUNK_BYTES);
    put_u32(out + 12, (uint32_t)nc);
    memcpy(out + 16, len, 256);
    for (uint64_t c = 0; c <= nc; c++) put_u32(out + 272 + 4 * c, off[c]);
    memcpy(out + hdr, payload, words * 4);
    free(payload);
  }
  free(off);
  return hdr + words * 4;
}

int or_huffman_decode(const uint8_t* in, uint64_t inlen, uint8_t* G, uint64_t S) {
  uint8_t len[256];
  int count[17] = {0};
  uint32_t first_code[18];
  int first_index[18], sorted[256], nsorted = 0;
  if (inlen < 272) return OR_ERR_CORRUPT;
  uint64_t orig = get_u64(in), nc = get_u32(in + 12);
  if (orig != S || get_u32(in + 8) != OR_CHUNK_BYTES || nc != nchunks_of(S)) return OR_ERR_CORRUPT;
  uint64_t hdr = huffman_header_bytes(nc);
  if (inlen < hdr) return OR_ERR_CORRUPT;
  memcpy(len, in + 16, 256);
  for (int s = 0; s < 256; s++) {
    if (len[s] > 16) return OR_ERR_CORRUPT;
    if (len[s]) count[len[s]]++;
  }
  /* canonical decoding tables: first code and first sorted index per length */
  uint32_t c = 0;
  for (int L = 1; L <= 16; L++) {
    c = (c + (uint32_t)(L > 1 ? count[L - 1] : 0)) << (L > 1 ? 1 : 0);
    first_code[L] = c;
    first_index[L] = nsorted;
    for (int s = 0; s < 256; s++)
      if (len[s] == L) sorted[nsorted++] = s;
  }
  uint64_t words = (inlen - hdr) / 4;
  for (uint64_t ch = 0; ch < nc; ch++) {
    uint64_t w0 = get_u32(in + 272 + 4 * ch), w1 = get_u32(in + 272 + 4 * (ch + 1));
    if (w0 > w1 || w1 > words) return OR_ERR_CORRUPT;
    uint64_t pos = w0 * 32, lim = w1 * 32;
    uint64_t end = (ch + 1) * OR_CHUNK_BYTES < S ? (ch + 1) * OR_CHUNK_BYTES : S;
    for (uint64_t i = ch * OR_CHUNK_BYTES; i < end; i++) {
      uint32_t code = 0;
      int L, found = -1;
      for (L = 1; L <= 16; L++) {
        if (pos >= lim) return OR_ERR_CORRUPT;
        uint32_t word = get_u32(in + hdr + 4 * (pos >> 5));
        code = (code << 1) | ((word >> (31 - (pos & 31))) & 1u);
        pos++;
        if (count[L] && code >= first_code[L] && code - first_code[L] < (uint32_t)count[L]) {
          found = sorted[first_index[L] + (int)(code - first_code[L])];
          break;
        }
      }
      if (found < 0) return OR_ERR_CORRUPT;
      G[i] = (uint8_t)found;
    }
  }
  return OR_OK;
}

/* -------------------------------------------------------------------- RLE */

static int leb_len(uint64_t v) {
  int n = 1;
  while (v >= 128) {
    v >>= 7;
    n++;
  }
  return n;
}

static uint64_t rle_header_bytes(uint64_t nchunks) { return 8 + 4 + 4 + 4 * (nchunks + 1); }

/* payload bytes of one chunk, written to out when out != NULL */
static uint64_t rle_chunk(const uint8_t* G, uint64_t a, uint64_t b, uint8_t* out) {
  uint64_t i = a, o = 0;
  while (i < b) {
    uint8_t v = G[i];
    uint64_t r = 1;
    while (i + r < b && G[i + r] == v) r++;
    if (out) out[o] = v;
    o++;
    uint64_t x = r - 1;
    while (x >= 128) {
      if (out) out[o] = (uint8_t)((x & 127) | 128);
      o++;
      x >>= 7;
    }
    if (out) out[o] = (uint8_t)x;
    o++;
    i += r;
  }
  return o;
}

uint64_t or_rle_estimate(const uint8_t* G, uint64_t S) {
  uint64_t nc = nchunks_of(S), total = rle_header_bytes(nc);
  for (uint64_t c = 0; c < nc; c++) {
    uint64_t a = c * OR_CHUNK_BYTES, b = a + OR_CHUNK_BYTES < S ? a + OR_CHUNK_BYTES : S;
    /* sum over runs of (1 + LEB128 length of run-1) */
    uint64_t i = a;
    while (i < b) {
      uint64_t r = 1;
      while (i + r < b && G[i + r] == G[i]) r++;
      total += 1 + (uint64_t)leb_len(r - 1);
      i += r;
    }
  }
  return total;
}

uint64_t or_rle_encode(const uint8_t* G, uint64_t S, uint8_t* out) {
  uint64_t nc = nchunks_of(S), hdr = rle_header_bytes(nc), o = 0;
  for (uint64_t c = 0; c < nc; c++) {
    uint64_t a = c * OR_CHUNK_BYTES, b = a + OR_CHUNK_BYTES < S ? a + OR_CHUNK_BYTES : S;
    if (out) put_u32(out + 16 + 4 * c, (uint32_t)o);
    o += rle_chunk(G, a, b, out ? out + hdr + o : NULL);
  }
  if (out) {
    put_u64(out, S);
    put_u32(out + 8, OR_CHUNK_BYTES);
    put_u32(out + 12, (uint32_t)nc);
    put_u32(out + 16 + 4 * nc, (uint32_t)o);
  }
  return hdr + o;
}

int or_rle_decode(const uint8_t* in, uint64_t inlen, uint8_t* G, uint64_t S) {
  if (inlen < 16) return OR_ERR_CORRUPT;
  uint64_t nc = get_u32(in + 12);
  if (get_u64(in) != S || get_u32(in + 8) != OR_CHUNK_BYTES || nc != nchunks_of(S))
    return OR_ERR_CORRUPT;
  uint64_t hdr = rle_header_bytes(nc);
  if (inlen < hdr) return OR_ERR_CORRUPT;
  for (uint64_t c = 0; c < nc; c++) {
    uint64_t p = get_u32(in + 16 + 4 * c), pe = get_u32(in + 16 + 4 * (c + 1));
    uint64_t a = c * OR_CHUNK_BYTES, b = a + OR_CHUNK_BYTES < S ? a + OR_CHUNK_BYTES : S;
    uint64_t i = a;
    if (p > pe || hdr + pe > inlen) return OR_ERR_CORRUPT;
    while (p < pe) {
      uint8_t v = in[hdr + p++];
      uint64_t x = 0;
      int shift = 0;
      for (;;) {
        if (p >= pe || shift > 56) return OR_ERR_CORRUPT;
        uint8_t byte = in[hdr + p++];
        x |= (uint64_t)(byte & 127) << shift;
        shift += 7;
        if (!(byte & 128)) break;
      }
      if (x + 1 > b - i) return OR_ERR_CORRUPT;
      for (uint64_t r = 0; r <= x; r++) G[i++] = v;
    }
    if (i != b) return OR_ERR_CORRUPT;
  }
  return OR_OK;
}

/* ------------------------------------------------------------- Algorithm 2 */

int or_hybrid_choose(uint64_t S, uint64_t est_H, uint64_t est_R, const or_hybrid_cfg* c) {
  if (S > c->Ts) {
    if ((u128)S * c->cr_den > (u128)c->cr_num * est_H) return OR_HUFFMAN;
    if ((u128)S * c->cr_den > (u128)c->cr_num * est_R) return OR_RLE;
    return OR_DC;
  }
  return OR_DC;
}

uint64_t or_hybrid_encode(const uint8_t* G, uint64_t S, const or_hybrid_cfg* c, int* method,
                          uint8_t* out) {
  uint64_t hist[256];
  uint8_t len[256];
  or_histogram(G, S, hist);
  or_huffman_lengths(hist, len);
  uint64_t est_H = or_huffman_estimate(hist, len, S);
  uint64_t est_R = or_rle_estimate(G, S);
  *method = or_hybrid_choose(S, est_H, est_R, c);
  if (*method == OR_HUFFMAN) return or_huffman_encode(G, S, out);
  if (*method == OR_RLE) return or_rle_encode(G, S, out);
  if (out) memcpy(out, G, S);
  return S;
}
