/*
 * Oracle: end-to-end refactor and retrieve, composed from the step functions
 * in the order of the paper's pipeline (Sec. 3, Fig. "framework"):
 * decompose -> align + Algorithm 1 -> Algorithm 2 per merged group; and for
 * retrieval: select groups for the bound -> lossless decode -> bitplane
 * decode -> recompose.  TEST INFRASTRUCTURE ONLY (see hpmdr_oracle.h).
 * Every retrieval starts from the stored bytes; nothing is cached.
 */
#include <stdlib.h>
#include <string.h>

#include "hpmdr_oracle.h"

#define OR_MAX_GROUPS 16

typedef struct or_field {
  int dtype, B, nlev, E_f, input_exact;
  uint64_t dims[3];
  or_stats st;
  or_hybrid_cfg cfg;
  uint64_t n[OR_MAX_LEVELS], W[OR_MAX_LEVELS];
  int bl[OR_MAX_LEVELS], exact[OR_MAX_LEVELS];
  uint32_t* planes[OR_MAX_LEVELS];
  int method[OR_MAX_LEVELS][OR_MAX_GROUPS];
  uint64_t est_H[OR_MAX_LEVELS][OR_MAX_GROUPS], est_R[OR_MAX_LEVELS][OR_MAX_GROUPS];
  uint64_t stored_len[OR_MAX_LEVELS][OR_MAX_GROUPS];
  uint8_t* stored[OR_MAX_LEVELS][OR_MAX_GROUPS];
} or_field;

void or_field_free(or_field* F) {
  if (!F) return;
  for (int l = 0; l < F->nlev; l++) {
    free(F->planes[l]);
    for (int g = 0; g < or_num_groups(F->B); g++) free(F->stored[l][g]);
  }
  free(F);
}

or_field* or_refactor(const void* f, const uint64_t dims[3], int dtype, const or_hybrid_cfg* cfg,
                      int* status) {
  or_field* F = (or_field*)calloc(1, sizeof(or_field));
  uint64_t N = dims[0] * dims[1] * dims[2];
  F->dtype = dtype;
  F->B = dtype == OR_F32 ? 32 : 64;
  memcpy(F->dims, dims, sizeof(F->dims));
  F->cfg = *cfg;
  F->nlev = or_num_levels(dims);
  *status = or_field_stats(f, N, dtype, &F->st);
  if (*status != OR_OK || F->nlev > OR_MAX_LEVELS) {
    if (*status == OR_OK) *status = OR_ERR_ARG;
    free(F);
    return NULL;
  }
  F->E_f = F->st.E_f;
  F->input_exact = F->st.input_exact;
  for (int l = 0; l < F->nlev; l++) {
    uint64_t n = or_level_size(dims, l), W = or_plane_words(n);
    int64_t* C8 = (int64_t*)malloc(n * sizeof(int64_t));
    uint64_t* q = (uint64_t*)malloc(n * sizeof(uint64_t));
    uint8_t* s = (uint8_t*)malloc(n);
    F->n[l] = n;
    F->W[l] = W;
    or_level_coeffs(f, dims, dtype, F->E_f, l, C8);
    F->bl[l] = or_bitlen_max(C8, n);
    or_quantize(C8, n, F->B, F->bl[l], q, s);
    F->exact[l] = or_level_exact(C8, n, F->B, F->bl[l]);
    F->planes[l] = (uint32_t*)malloc((size_t)(F->B + 1) * W * 4);
    or_bitplane_encode(q, s, n, F->B, F->planes[l]);
    for (int g = 0; g < or_num_groups(F->B); g++) {
      const uint8_t* G = (const uint8_t*)F->planes[l] + or_group_offset(W, g);
      uint64_t S = or_group_size(W, g), hist[256];
      uint8_t len[256];
      or_histogram(G, S, hist);
      or_huffman_lengths(hist, len);
      F->est_H[l][g] = or_huffman_estimate(hist, len, S);
      F->est_R[l][g] = or_rle_estimate(G, S);
      int m;
      uint64_t sz = or_hybrid_encode(G, S, cfg, &m, NULL);
      F->stored[l][g] = (uint8_t*)malloc(sz);
      (void)or_hybrid_encode(G, S, cfg, &m, F->stored[l][g]);
      F->method[l][g] = m;
      F->stored_len[l][g] = sz;
    }
    free(C8);
    free(q);
    free(s);
  }
  return F;
}

/* metadata the selection sees */
static void sel_meta(const or_field* F, or_sel_meta* m) {
  memset(m, 0, sizeof(*m));
  m->nlev = F->nlev;
  m->B = F->B;
  m->dtype = F->dtype;
  m->E_f = F->E_f;
  m->input_exact = F->input_exact;
  for (int l = 0; l < F->nlev; l++) {
    m->bl[l] = F->bl[l];
    m->exact[l] = F->exact[l];
    m->ngroups[l] = or_num_groups(F->B);
    m->group_bytes[l] = F->stored_len[l];
  }
}

int or_field_select(const or_field* F, double tau_abs, int* g, double* E_abs, uint64_t* E_hi,
                    uint64_t* E_lo) {
  or_sel_meta m;
  sel_meta(F, &m);
  return or_select(&m, tau_abs, g, E_abs, E_hi, E_lo);
}

void or_field_estimate(const or_field* F, const int* g, double* E_abs) {
  or_sel_meta m;
  sel_meta(F, &m);
  uint64_t hi, lo;
  or_estimate(&m, g, &hi, &lo);
  *E_abs = or_units_to_abs(hi, lo, F->E_f, F->B);
}

int or_field_sequence(const or_field* F, int* seq, int cap) {
  or_sel_meta m;
  sel_meta(F, &m);
  return or_greedy_sequence(&m, seq, cap);
}

/* reconstruct from the first g[l] groups of each level, decoding stored bytes */
int or_reconstruct(const or_field* F, const int* g, void* out) {
  int64_t* c8hat[OR_MAX_LEVELS] = {0};
  int rc = OR_OK;
  for (int l = 0; l < F->nlev; l++) {
    uint64_t n = F->n[l], W = F->W[l];
    uint32_t* planes = (uint32_t*)calloc((size_t)(F->B + 1) * W, 4);
    uint64_t* q = (uint64_t*)malloc(n * sizeof(uint64_t));
    uint8_t* s = (uint8_t*)malloc(n);
    for (int gi = 0; gi < g[l]; gi++) {
      uint8_t* G = (uint8_t*)planes + or_group_offset(W, gi);
      uint64_t S = or_group_size(W, gi);
      int m = F->method[l][gi];
      if (m == OR_HUFFMAN) rc |= or_huffman_decode(F->stored[l][gi], F->stored_len[l][gi], G, S);
      else if (m == OR_RLE) rc |= or_rle_decode(F->stored[l][gi], F->stored_len[l][gi], G, S);
      else memcpy(G, F->stored[l][gi], S);
    }
    or_bitplane_decode(planes, n, F->B, 4 * g[l], q, s);
    c8hat[l] = (int64_t*)malloc(n * sizeof(int64_t));
    for (uint64_t j = 0; j < n; j++) c8hat[l][j] = or_dequantize(q[j], s[j], F->B, F->bl[l]);
    free(planes);
    free(q);
    free(s);
  }
  or_recompose(F->dims, F->dtype, F->E_f, (const int64_t* const*)c8hat, out);
  for (int l = 0; l < F->nlev; l++) free(c8hat[l]);
  return rc ? OR_ERR_CORRUPT : OR_OK;
}

int or_retrieve(const or_field* F, double tau_abs, void* out, int* g, double* E_abs,
                uint64_t* E_hi, uint64_t* E_lo) {
  int status = or_field_select(F, tau_abs, g, E_abs, E_hi, E_lo);
  int rc = or_reconstruct(F, g, out);
  return rc != OR_OK ? rc : status;
}

/* ---- accessors ---------------------------------------------------------- */
void or_field_info(const or_field* F, int* nlev, int* E_f, int* input_exact, double stats[4]) {
  *nlev = F->nlev;
  *E_f = F->E_f;
  *input_exact = F->input_exact;
  stats[0] = F->st.maxabs;
  stats[1] = F->st.vmin;
  stats[2] = F->st.vmax;
  stats[3] = F->st.range;
}

void or_field_level(const or_field* F, int l, uint64_t* n, int* bl, int* exact) {
  *n = F->n[l];
  *bl = F->bl[l];
  *exact = F->exact[l];
}

const uint32_t* or_field_planes(const or_field* F, int l) { return F->planes[l]; }

const uint8_t* or_field_group(const or_field* F, int l, int g, uint64_t* len, int* method,
                              uint64_t est[2]) {
  *len = F->stored_len[l][g];
  *method = F->method[l][g];
  est[0] = F->est_H[l][g];
  est[1] = F->est_R[l][g];
  return F->stored[l][g];
}
