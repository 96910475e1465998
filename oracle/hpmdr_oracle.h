/*
 * Plain CPU oracle for the HP-MDR progressive-refactoring hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library and its Python binding) never calls it, and the two share
 * no code, headers, tables or constants.
 *
 * Every function is written step by step from the paper (HP-MDR, arXiv
 * 2505.00227): Algorithm 1 (bitplane encoding, Sec. 4), Algorithm 2 (hybrid
 * lossless compression, Sec. 5.2) with its Huffman and RLE ratio estimators,
 * the error-controlled retrieval of Sec. 3 / Sec. 6.2 and Algorithm 3.  Where
 * the paper gives no definition (the multilevel decomposer, coefficient order,
 * bit layout, coder formats, the error estimator and the greedy selection),
 * the reading documented beside each function is used.  Integer arithmetic is
 * exact; floating point is used only where the reading says so, compiled with
 * -ffp-contract=off.
 */
#ifndef HPMDR_ORACLE_H
#define HPMDR_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_F32 = 0, OR_F64 = 1 };
enum { OR_DC = 0, OR_HUFFMAN = 1, OR_RLE = 2, OR_PLACEHOLDER = 3 };
enum { OR_OK = 0, OR_ERR_ARG = -1, OR_ERR_CORRUPT = -4, OR_ERR_UNATTAINABLE = -5 };

#define OR_CHUNK_BYTES 16384u  /* coder input chunk (Huffman and RLE) */
#define OR_MAX_LEVELS 64

/* ---- level geometry (multilevel decomposition, Sec. 3) ---------------- */
int      or_num_levels(const uint64_t dims[3]);           /* root + details */
uint64_t or_level_size(const uint64_t dims[3], int l);    /* nodes in level l */
uint64_t or_plane_words(uint64_t n);                      /* 4*ceil(n/128) */

/* ---- field statistics (alignment prerequisite, Sec. 4) ------------------ */
typedef struct {
  double maxabs, vmin, vmax, range;
  int E_f;          /* smallest integer with max|f| < 2^E_f (0 for a zero field) */
  int input_exact;  /* every f_i is an integer multiple of U = 2^(E_f-48) */
} or_stats;
int or_field_stats(const void* f, uint64_t N, int dtype, or_stats* st);

/* F_i = sign(f_i) * floor(|f_i| / 2^(E_f-48)), exact from the IEEE bits */
int64_t or_fixed_point(const void* f, uint64_t i, int dtype, int E_f, int* floored);

/* ---- multilevel decomposition: coefficients of one level ---------------- */
/* C8 in units of U/8, in the level's linear order (parity types 1..7,
 * raster order inside a type).  Level 0 is the root (one node). */
void or_level_coeffs(const void* f, const uint64_t dims[3], int dtype, int E_f,
                     int l, int64_t* C8);


/* ---- exponent alignment + Algorithm 1 ----------------------------------- */
int  or_bitlen_max(const int64_t* C8, uint64_t n);          /* bl = bitlen(max|C8|) */
void or_quantize(const int64_t* C8, uint64_t n, int B, int bl, uint64_t* q, uint8_t* sign);
int  or_level_exact(const int64_t* C8, uint64_t n, int B, int bl);
/* planes: (B+1) planes of W=or_plane_words(n) uint32 words; plane 0 = sign,
 * plane 1+p = magnitude bit B-1-p (Alg. 1 runs b = B-1 .. 0). */
void or_bitplane_encode(const uint64_t* q, const uint8_t* sign, uint64_t n, int B,
                        uint32_t* planes);
/* inverse: top-k magnitude planes (and the sign plane) -> q_hat, sign */
void or_bitplane_decode(const uint32_t* planes, uint64_t n, int B, int k,
                        uint64_t* q_hat, uint8_t* sign);

/* groups of m=4 planes: group 0 = sign + p0..p3, group g>=1 = p4g..p4g+3 */
int      or_num_groups(int B);
uint64_t or_group_offset(uint64_t W, int g);   /* byte offset of G_g in the plane buffer */
uint64_t or_group_size(uint64_t W, int g);     /* S = bytes of G_g */

/* ---- lossless coders (Sec. 5.1) ----------------------------------------- */
void     or_histogram(const uint8_t* G, uint64_t S, uint64_t hist[256]);
void     or_huffman_lengths(const uint64_t hist[256], uint8_t len[256]);
uint64_t or_huffman_estimate(const uint64_t hist[256], const uint8_t len[256], uint64_t S);
uint64_t or_huffman_encode(const uint8_t* G, uint64_t S, uint8_t* out);  /* out NULL: size */
int      or_huffman_decode(const uint8_t* in, uint64_t len, uint8_t* G, uint64_t S);
uint64_t or_rle_estimate(const uint8_t* G, uint64_t S);                  /* exact size */
uint64_t or_rle_encode(const uint8_t* G, uint64_t S, uint8_t* out);      /* out NULL: size */
int      or_rle_decode(const uint8_t* in, uint64_t len, uint8_t* G, uint64_t S);

/* ---- Algorithm 2: hybrid choice for one group --------------------------- */
typedef struct { uint64_t Ts; uint32_t cr_num, cr_den; } or_hybrid_cfg;
int or_hybrid_choose(uint64_t S, uint64_t est_H, uint64_t est_R, const or_hybrid_cfg* c);
/* encode G with the chosen method; returns stored length (out NULL: size) */
uint64_t or_hybrid_encode(const uint8_t* G, uint64_t S, const or_hybrid_cfg* c,
                          int* method, uint8_t* out);

/* ---- error estimator + greedy selection --------------------------------- */
typedef struct {
  int nlev, B, dtype, E_f, input_exact;
  int bl[OR_MAX_LEVELS];
  int exact[OR_MAX_LEVELS];
  int ngroups[OR_MAX_LEVELS];
  const uint64_t* group_bytes[OR_MAX_LEVELS];   /* stored bytes per group */
} or_sel_meta;
/* estimate E (units of 2^(E_f-51-B)) for g[l] groups per level, as hi/lo words */
void or_estimate(const or_sel_meta* m, const int* g, uint64_t* E_hi, uint64_t* E_lo);
/* greedy sequence: seq[i] = level picked at step i; returns its length */
int  or_greedy_sequence(const or_sel_meta* m, int* seq, int cap);
/* tau_abs -> g[] (smallest prefix with E <= tau); returns OR_OK or
 * OR_ERR_UNATTAINABLE (g = everything).  E reported in absolute units. */
int  or_select(const or_sel_meta* m, double tau_abs, int* g, double* E_abs,
               uint64_t* E_hi, uint64_t* E_lo);
double or_units_to_abs(uint64_t hi, uint64_t lo, int E_f, int B);
void   or_tau_units(double tau_abs, int E_f, int B, uint64_t* hi, uint64_t* lo);

/* ---- recomposition ------------------------------------------------------ */
/* c8hat[l] = reconstructed coefficients of level l (NULL = all zero) */
void or_recompose(const uint64_t dims[3], int dtype, int E_f,
                  const int64_t* const* c8hat, void* out);
/* coefficient from the fetched top bits of q: truncation, no midpoint */
int64_t or_dequantize(uint64_t qhat, int s, int B, int bl);

/* ---- QoI: velocity magnitude ------------------------------------------- */
float or_vmag(float x, float y, float z);
void  or_vmag_field(const float* vx, const float* vy, const float* vz, uint64_t N,
                    float* out, float* qmin, float* qmax);
double or_qoi_component_bound(double tau_q_abs, double qmax);
double or_qoi_estimate(double Ex, double Ey, double Ez, double qmax);

/* ---- end-to-end composition (pipeline.c) ------------------------------- */
typedef struct or_field or_field;
or_field* or_refactor(const void* f, const uint64_t dims[3], int dtype, const or_hybrid_cfg* cfg,
                      int* status);
void      or_field_free(or_field* F);
int       or_field_select(const or_field* F, double tau_abs, int* g, double* E_abs,
                          uint64_t* E_hi, uint64_t* E_lo);
int       or_field_sequence(const or_field* F, int* seq, int cap);
int       or_reconstruct(const or_field* F, const int* g, void* out);
int       or_retrieve(const or_field* F, double tau_abs, void* out, int* g, double* E_abs,
                      uint64_t* E_hi, uint64_t* E_lo);
void      or_field_info(const or_field* F, int* nlev, int* E_f, int* input_exact, double stats[4]);
void      or_field_level(const or_field* F, int l, uint64_t* n, int* bl, int* exact);
const uint32_t* or_field_planes(const or_field* F, int l);
const uint8_t*  or_field_group(const or_field* F, int l, int g, uint64_t* len, int* method,
                               uint64_t est[2]);

/* Estimate (absolute) of the first g[l] groups of every level */
void      or_field_estimate(const or_field* F, const int* g, double* E_abs);

/* ---- QoI: total velocity V = vx^2 + vy^2 + vz^2, iterated (qoi_iter.c) -- */
enum { OR_EST_CP = 0, OR_EST_MA = 1, OR_EST_MAPE = 2 };
#define OR_QOI_MAX_ITERATIONS 4096
#define OR_QOI_MAX_HALVINGS 1100
typedef struct {
  int status, iterations;
  double tau_abs, est, eps[3];     /* requested, final QoI bound, final data estimates */
  int prefix[3];                   /* sequence steps retrieved per variable */
  int g[3][OR_MAX_LEVELS];         /* groups per level per variable */
} or_qoi_report;
double or_vtotal(float x, float y, float z);
void   or_vtotal_range(const float* vx, const float* vy, const float* vz, uint64_t N,
                       double* vmin, double* vmax);
double or_vtotal_point_bound(float x, float y, float z, const double e[3]);
double or_vtotal_bound(const float* x, const float* y, const float* z, uint64_t N,
                       const double e[3], uint64_t* arg);
double or_field_prefix_estimate(const or_field* F, int k);
int    or_qoi_vtotal(const or_field* const F[3], uint64_t N, double vt_min, double vt_max,
                     double tau_rel, int estimator, double c, float* out[3], float* qoi,
                     or_qoi_report* rep);

#ifdef __cplusplus
}
#endif
#endif
