/*
 * Oracle: field statistics, exact fixed-point multilevel decomposition and
 * recomposition.  TEST INFRASTRUCTURE ONLY (see hpmdr_oracle.h).
 *
 * The paper names a multilevel decomposer (Sec. 3, Fig. "framework") and
 * aligns every element of a decomposed array to the maximum exponent before
 * bitplane encoding (Sec. 4, Algorithm 1, "AlignExponent"), but gives no
 * equations for the decomposition.  The reading implemented here:
 *   - interpolation-only hierarchical basis: coefficient = value minus the
 *     multilinear interpolant of the next-coarser grid;
 *   - levels by half-stride h = h_max .. 1, h_max the largest power of two
 *     below max_d n_d; a node belongs to level h iff all of its coordinates are
 *     multiples of h and not all are multiples of 2h; the root is node (0,0,0);
 *   - along an odd axis the neighbours are i-h and i+h, and a right neighbour
 *     outside the grid is replaced by the left one;
 *   - exact integer arithmetic: F = sign(f) * floor(|f| / U), U = 2^(E_f-48),
 *     D = k*F_i - sum of the k = 2^|odd axes| corners, C8 = D * 8/k (units U/8);
 *   - inside a level, parity type t = o_x + 2 o_y + 4 o_z for t = 1..7, raster
 *     order (z outer, x inner) inside a type.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "hpmdr_oracle.h"

/* ---------------------------------------------------------------- geometry */

static uint64_t max3(const uint64_t d[3]) {
  uint64_t m = d[0];
  if (d[1] > m) m = d[1];
  if (d[2] > m) m = d[2];
  return m;
}

/* number of detail levels L: h_max = 2^(L-1) is the largest power of two
 * strictly below max_d n_d; a single-node field has no detail level */
static int num_detail_levels(const uint64_t dims[3]) {
  uint64_t n = max3(dims);
  int L = 0;
  uint64_t h = 1;
  if (n <= 1) return 0;
  while (h < n) { /* count h = 1, 2, 4, ... while h < n */
    L++;
    h *= 2;
  }
  return L;
}

int or_num_levels(const uint64_t dims[3]) { return num_detail_levels(dims) + 1; }

static uint64_t half_stride(const uint64_t dims[3], int l) {
  int L = num_detail_levels(dims);
  return (uint64_t)1 << (L - l);
}

/* nodes of one parity along an axis of the level grid: o = 0 even, o = 1 odd */
static uint64_t axis_count(uint64_t n_grid, int o) {
  return o ? n_grid / 2 : (n_grid + 1) / 2;
}

uint64_t or_level_size(const uint64_t dims[3], int l) {
  uint64_t h, g[3], total = 0;
  int t;
  if (l == 0) return 1;
  h = half_stride(dims, l);
  for (int d = 0; d < 3; d++) g[d] = (dims[d] + h - 1) / h;
  for (t = 1; t < 8; t++) {
    int ox = t & 1, oy = (t >> 1) & 1, oz = (t >> 2) & 1;
    total += axis_count(g[0], oz) * axis_count(g[1], oy) * axis_count(g[2], ox);
  }
  return total;
}

uint64_t or_plane_words(uint64_t n) { return 4 * ((n + 127) / 128); }

/* ------------------------------------------------------------ statistics */

static int bitlen64(uint64_t v) {
  int b = 0;
  while (v) {
    b++;
    v >>= 1;
  }
  return b;
}

static double value_at(const void* f, uint64_t i, int dtype) {
  if (dtype == OR_F32) return (double)((const float*)f)[i];
  return ((const double*)f)[i];
}

/* E_f = smallest integer E with max|f| < 2^E, read from the IEEE fields */
static int exponent_bound(double maxabs, int dtype) {
  if (maxabs == 0.0) return 0;
  if (dtype == OR_F32) {
    float m = (float)maxabs;
    uint32_t u;
    memcpy(&u, &m, 4);
    int e = (int)((u >> 23) & 0xff);
    if (e == 0) return bitlen64(u & 0x7fffffu) - 149;
    return e - 126;
  } else {
    uint64_t u;
    memcpy(&u, &maxabs, 8);
    int e = (int)((u >> 52) & 0x7ff);
    if (e == 0) return bitlen64(u & 0xfffffffffffffull) - 1074;
    return e - 1022;
  }
}

int64_t or_fixed_point(const void* f, uint64_t i, int dtype, int E_f, int* floored) {
  uint64_t m, mag;
  int neg, e_eff, s;
  if (dtype == OR_F32) {
    uint32_t u;
    memcpy(&u, (const float*)f + i, 4);
    neg = (int)(u >> 31);
    e_eff = (int)((u >> 23) & 0xff);
    m = u & 0x7fffffu;
    if (e_eff == 0) e_eff = 1; else m |= 0x800000u;
    s = e_eff - 150 - (E_f - 48); /* |f| = m 2^(e_eff-150), U = 2^(E_f-48) */
  } else {
    uint64_t u;
    memcpy(&u, (const double*)f + i, 8);
    neg = (int)(u >> 63);
    e_eff = (int)((u >> 52) & 0x7ff);
    m = u & 0xfffffffffffffull;
    if (e_eff == 0) e_eff = 1; else m |= 0x10000000000000ull;
    s = e_eff - 1075 - (E_f - 48);
  }
  if (s >= 0) {
    mag = m << s;
    if (floored) *floored = 0;
  } else if (-s >= 64) {
    mag = 0;
    if (floored) *floored = (m != 0);
  } else {
    mag = m >> (-s);
    if (floored) *floored = ((m & ((1ull << (-s)) - 1)) != 0);
  }
  return neg ? -(int64_t)mag : (int64_t)mag;
}

int or_field_stats(const void* f, uint64_t N, int dtype, or_stats* st) {
  double mx = 0.0, lo = 0.0, hi = 0.0;
  int exact = 1;
  for (uint64_t i = 0; i < N; i++) {
    double v = value_at(f, i, dtype);
    if (!(v == v) || isinf(v)) return OR_ERR_ARG;
    if (i == 0 || v < lo) lo = v;
    if (i == 0 || v > hi) hi = v;
    if (fabs(v) > mx) mx = fabs(v);
  }
  st->maxabs = mx;
  st->vmin = lo;
  st->vmax = hi;
  st->range = hi - lo;
  st->E_f = exponent_bound(mx, dtype);
  if (dtype == OR_F32 && st->E_f > 121) return OR_ERR_ARG;
  if (dtype == OR_F64 && (st->E_f > 1017 || (mx != 0.0 && st->E_f < -1000))) return OR_ERR_ARG;
  for (uint64_t i = 0; i < N && exact; i++) {
    int fl = 0;
    (void)or_fixed_point(f, i, dtype, st->E_f, &fl);
    if (fl) exact = 0;
  }
  st->input_exact = exact;
  return OR_OK;
}

/* ------------------------------------------------------- decomposition */

typedef struct {
  uint64_t i[3];        /* full-resolution coordinates (z, y, x) */
  int ncorner;          /* k = 2^|odd axes| */
  int nodd;
  uint64_t corner[8][3];
} stencil;

/* corners of node i at half-stride h: along odd axes i-h / i+h, with the
 * right neighbour replaced by the left one when it falls outside the grid */
static void make_stencil(const uint64_t dims[3], uint64_t h, const int odd[3], stencil* s) {
  uint64_t lo[3], hi[3];
  int axes[3], na = 0;
  for (int d = 0; d < 3; d++) {
    if (odd[d]) {
      lo[d] = s->i[d] - h;
      hi[d] = (s->i[d] + h < dims[d]) ? s->i[d] + h : s->i[d] - h;
      axes[na++] = d;
    } else {
      lo[d] = hi[d] = s->i[d];
    }
  }
  s->nodd = na;
  s->ncorner = 1 << na;
  for (int c = 0; c < s->ncorner; c++) {
    for (int d = 0; d < 3; d++) s->corner[c][d] = s->i[d];
    for (int a = 0; a < na; a++) {
      int d = axes[a];
      s->corner[c][d] = ((c >> a) & 1) ? hi[d] : lo[d];
    }
  }
}

static uint64_t lin(const uint64_t dims[3], const uint64_t i[3]) {
  return (i[0] * dims[1] + i[1]) * dims[2] + i[2];
}

/* visit the nodes of level l >= 1 in their linear order */
typedef void (*node_fn)(void* ctx, uint64_t j, const stencil* s);

static void for_each_node(const uint64_t dims[3], int l, node_fn fn, void* ctx) {
  uint64_t h = half_stride(dims, l), g[3], j = 0;
  for (int d = 0; d < 3; d++) g[d] = (dims[d] + h - 1) / h;
  for (int t = 1; t < 8; t++) {
    int odd[3] = {(t >> 2) & 1, (t >> 1) & 1, t & 1}; /* z, y, x */
    uint64_t cz = axis_count(g[0], odd[0]), cy = axis_count(g[1], odd[1]),
             cx = axis_count(g[2], odd[2]);
    for (uint64_t a = 0; a < cz; a++)
      for (uint64_t b = 0; b < cy; b++)
        for (uint64_t c = 0; c < cx; c++) {
          stencil s;
          s.i[0] = h * (2 * a + (uint64_t)odd[0]);
          s.i[1] = h * (2 * b + (uint64_t)odd[1]);
          s.i[2] = h * (2 * c + (uint64_t)odd[2]);
          make_stencil(dims, h, odd, &s);
          fn(ctx, j++, &s);
        }
  }
}

typedef struct {
  const void* f;
  const uint64_t* dims;
  int dtype, E_f;
  int64_t* C8;
} coeff_ctx;

static void coeff_node(void* vctx, uint64_t j, const stencil* s) {
  coeff_ctx* c = (coeff_ctx*)vctx;
  int64_t Fi = or_fixed_point(c->f, lin(c->dims, s->i), c->dtype, c->E_f, NULL);
  int64_t sum = 0, D;
  for (int k = 0; k < s->ncorner; k++)
    sum += or_fixed_point(c->f, lin(c->dims, s->corner[k]), c->dtype, c->E_f, NULL);
  D = (int64_t)s->ncorner * Fi - sum;
  c->C8[j] = D * (8 / s->ncorner); /* exact coefficient D/k in units of U/8 */
}

void or_level_coeffs(const void* f, const uint64_t dims[3], int dtype, int E_f, int l,
                     int64_t* C8) {
  if (l == 0) {
    uint64_t o[3] = {0, 0, 0};
    C8[0] = 8 * or_fixed_point(f, lin(dims, o), dtype, E_f, NULL);
    return;
  }
  coeff_ctx c = {f, dims, dtype, E_f, C8};
  for_each_node(dims, l, coeff_node, &c);
}

/* ------------------------------------------------------- recomposition */

/* floor(a / 2^s) for signed a, written without relying on >> of negatives */
static int64_t floor_div_pow2(int64_t a, int s) {
  int64_t d = (int64_t)1 << s;
  if (a >= 0) return a / d;
  return -((-a + d - 1) / d);
}

typedef struct {
  const uint64_t* dims;
  const int64_t* c8;
  int64_t* X;
} recomp_ctx;

static void recomp_node(void* vctx, uint64_t j, const stencil* s) {
  recomp_ctx* c = (recomp_ctx*)vctx;
  int64_t sum = 0, c8 = c->c8 ? c->c8[j] : 0;
  for (int k = 0; k < s->ncorner; k++) sum += c->X[lin(c->dims, s->corner[k])];
  /* X = floor((c8 * k + 8 * sum) / (8 k)); 8k = 2^(3 + |odd axes|) */
  c->X[lin(c->dims, s->i)] = floor_div_pow2(c8 * s->ncorner + 8 * sum, 3 + s->nodd);
}

static float to_f32(int64_t X, int E_f) {
  int e = E_f - 48;
  if (e >= -126 && E_f <= 121) {
    float y = (float)X;               /* one round-to-nearest conversion */
    return y * ldexpf(1.0f, e);       /* exact power-of-two scale */
  } else {
    double d = (double)X;
    d = d * ldexp(1.0, e);
    return (float)d;
  }
}

static double to_f64(int64_t X, int E_f) {
  int e = E_f - 48;
  double d = (double)X;
  if (e >= -1022) return d * ldexp(1.0, e);
  d = d * ldexp(1.0, -500);
  return d * ldexp(1.0, e + 500);
}

void or_recompose(const uint64_t dims[3], int dtype, int E_f, const int64_t* const* c8hat,
                  void* out) {
  uint64_t N = dims[0] * dims[1] * dims[2];
  int nlev = or_num_levels(dims);
  int64_t* X = (int64_t*)calloc(N, sizeof(int64_t));
  X[0] = floor_div_pow2(c8hat[0] ? c8hat[0][0] : 0, 3);
  for (int l = 1; l < nlev; l++) {
    recomp_ctx c = {dims, c8hat[l], X};
    for_each_node(dims, l, recomp_node, &c);
  }
  for (uint64_t i = 0; i < N; i++) {
    if (dtype == OR_F32) ((float*)out)[i] = to_f32(X[i], E_f);
    else ((double*)out)[i] = to_f64(X[i], E_f);
  }
  free(X);
}
