// Internal data structures shared by the host runtime and the sm_103a kernels.
//
// Layout in HBM of one refactored field (a "handle"):
//   planes   : for each level l, (B+1) bitplanes of W_l uint32 words, plane 0 =
//              sign, plane 1+p = magnitude bit B-1-p (Algorithm 1 order).  A
//              merged group (Sec. 5.2) is a contiguous byte range of it.  Groups
//              stored by direct copy live here; Huffman/RLE groups are decoded
//              back into their range on retrieval.
//   slots    : one fixed slot per (level, group) of capacity S*cr_den/cr_num
//              (+header room) for the Huffman or RLE bytes of that group.
//              A compacted handle packs every group's stored bytes here, DC
//              groups included, and its plane buffer becomes a cache that a
//              retrieval allocates and fills (DC groups by copying).
//   meta     : FieldMeta (device), mirrored to the host after refactor.
#pragma once
#include <cstddef>
#include <cstdint>

#define HP_MAX_LEVELS 33
#define HP_MAX_GROUPS 16
#define HP_CHUNK 16384u
#define HP_TILE 1024u  // level-linear elements per warp tile (32 words)
#define HP_SEQ_MAX (HP_MAX_LEVELS * HP_MAX_GROUPS)

// unsigned 32-bit division by a runtime constant (round-up multiplier method)
struct FastDiv {
  uint32_t d, m, s;  // q = (umulhi(n, m) + n) >> s  for d > 1
};

// generic levels up to this many nodes (after the root) are recomposed by the
// one-CTA kernel, a few tiles at a time, instead of a launch per level
constexpr uint32_t kSmallLevelNodes = 4096;

struct LevelDesc {
  uint64_t plane_off;  // byte offset of this level's planes in the plane buffer
  uint32_t n;          // nodes in the level
  uint32_t W;          // uint32 words per plane
  uint32_t tile0;      // first global tile of this level
  uint32_t ntiles;
  uint32_t gtile0;     // first slot of the level in the generic kernels (0 tiles when fast)
  int32_t fast;        // 1: fused cell kernels, 2: general cell kernels, 0: tile kernels
  int32_t level;       // l (0 = root)
  int32_t hlog;        // log2 of the half-stride h (-1 for the root)
  uint32_t g[3];       // level grid G_h dims (z, y, x): ceil(n_d / h)
  uint32_t gc[3];      // coarse grid G_2h dims: ceil(g_d / 2)
  uint32_t off[9];     // offset of parity type t (t = 1..7) in the level, off[8] = n
  uint32_t cnt[8][3];  // nodes of type t along (z, y, x)
  FastDiv dx[8], dy[8];  // per type t >= 1: divide by cnt[t][2], cnt[t][1]; [0]: by gc[2], gc[1]
};

struct GroupMeta {
  uint64_t S;           // raw bytes of the merged group
  uint64_t plane_off;   // byte offset of the group in the plane buffer
  uint64_t slot_off;    // byte offset of its slot in the slot buffer
  uint64_t cap;         // slot capacity
  uint64_t stored_len;  // stored bytes (DC: S)
  uint64_t est_H, est_R;
  uint32_t nchunks, chunk0;  // 16 KiB chunks and the global index of the first
  int32_t method;
  int32_t pad;
};

struct alignas(16) FieldMeta {
  int32_t status;  // HPMDR_OK or an error raised on the device
  int32_t dtype, B, nlev, ngroups, E_f, input_exact, has_range;
  uint64_t key_absmax, key_min, key_max;  // order-preserving keys of max|f|, min, max
  double maxabs, vmin, vmax, range;
  uint32_t floored;                       // some f_i lost bits in the fixed point
  // least exponent e of a set bit (weight 2^e) over the values the fused
  // statistics pass saw (INT32_MAX: none); some value loses bits in the fixed
  // point exactly when lsb_min < E_f - 48
  int32_t lsb_min;
  uint64_t m8[HP_MAX_LEVELS];             // max |C8| per level
  uint64_t lowbits[HP_MAX_LEVELS];        // OR of the bits dropped by alignment
  uint32_t m8est[HP_MAX_LEVELS];          // FP32 bits of max |detail| from the estimate pass
  int32_t bl[HP_MAX_LEVELS], exact[HP_MAX_LEVELS];
  GroupMeta grp[HP_MAX_LEVELS][HP_MAX_GROUPS];
  // greedy sequence and the estimate after each prefix (128-bit units)
  int32_t seq_len, pad1;
  uint8_t seq[HP_SEQ_MAX];
  uint64_t E_hi[HP_SEQ_MAX + 1], E_lo[HP_SEQ_MAX + 1];
  // retrieval state
  int32_t fetched[HP_MAX_LEVELS];  // groups present in the plane buffer per level
  int32_t cur[HP_MAX_LEVELS];      // groups used by the current reconstruction
  // QoI triplet data (velocity magnitude range) when prepared
  float qmin, qmax;
  // 1: every group (DC included) is read from the slot buffer on retrieval
  int32_t compact;
  // set by the selection of the current retrieval: 1 when its error bound
  // proves |X| < 2^48 for every reconstructed value X (max|f| + E < 2^E_f),
  // so the output conversion needs no per-value range test
  int32_t out_small;
};

// retrieval info written by the selection kernel
struct alignas(16) RetrieveDev {
  int32_t status, nsel;
  uint64_t E_hi, E_lo;
  double E_abs, tau_abs;
  uint64_t bytes_new, bytes_total;
  uint32_t n_new;                     // groups newly fetched by this retrieval
  uint32_t items;                     // Huffman/RLE chunks to decode
  int32_t g[HP_MAX_LEVELS];           // groups used per level
  uint32_t new_gi[HP_SEQ_MAX];        // flat index of each newly fetched coded group
  uint32_t new_pref[HP_SEQ_MAX + 1];  // prefix of their chunk counts
};

// --------------------------------------------------------- batched launches
// One field of a batched launch: every pointer the stage kernels of one field
// need.  A batched kernel runs over the work units of all its jobs (tiles,
// chunks, groups ... of every field); job j owns units [unit0[j], unit0[j+1]).
struct BatchJob {
  const void* f;  // field (device, 16-byte aligned)
  uint64_t N;
  uint32_t dims[3];
  uint32_t nlev, ngt, generic_tiles, total_chunks, pad0;
  FieldMeta* meta;
  const FieldMeta* meta0;  // the plan's initial metadata
  uint8_t* planes;
  uint8_t* slots;
  const LevelDesc* levels;
  const uint32_t* perm;
  const uint32_t* chunk_group;
  // refactor scratch: group histograms (256 per group), group RLE sizes,
  // chunk RLE costs, chunk Huffman words, chunk output offsets, code lengths
  uint32_t* hist;
  unsigned long long* gcost;
  uint32_t* ccost;
  uint32_t* cwords;
  uint32_t* cout;
  uint8_t* lens;
  // retrieval
  RetrieveDev* rd;
  int64_t* xroot;
  int64_t* xa;
  int64_t* xb;
  void* out;
  void* gq;          // staging of the general cell levels: aligned integers
  uint8_t* gsg;      // and signs
  double tau;        // relative L-infinity bound
  int32_t small_end;  // last level recomposed by the one-CTA small-level kernel
  int32_t pad1;
};

// (job, level) entry of a level-granular batched launch
struct LevelRef {
  uint32_t job, level;
  const int64_t* coarse;  // recomposition: the coarse grid G_2h
  int64_t* dst;           // recomposition: the level grid (unused when final)
  int32_t final;          // recomposition: the level writes the job's output
  int32_t pad;
  uint64_t soff;          // general cell levels: first element of the level's staging
};

// launchers implemented in the .cu files --------------------------------------
typedef struct CUstream_st* cstream;

namespace hp {

// counts every kernel launch made by the library (runtime.cu)
void note_launch();
// takes back launches counted while a CUDA graph was being captured
void unnote_launches(uint64_t k);
// raises a kernel's dynamic shared memory limit once per device (thread-safe)
void set_smem_once(const void* func, int bytes);

// stats.cu
void launch_meta_init(FieldMeta* meta, int dtype, int B, int nlev, int ngroups, cstream s);
// word copies (sizes multiples of 4 bytes) into mapped page-locked host memory
// by a one-CTA kernel; b and d are device pointers of the host buffers
void launch_to_host(const void* a, void* b, size_t na_bytes, const void* c, void* d,
                    size_t nc_bytes, cstream s);
void launch_stats(const void* f, uint64_t N, int dtype, FieldMeta* meta, cstream s);
void launch_stats_finalize(FieldMeta* meta, cstream s);

// decompose.cu
// perm: per level, the order in which its 1024-node tiles are processed (tiles
// of the 7 parity types covering the same region of the grid run together)
void launch_levelmax(const void* f, int dtype, const uint64_t dims[3], const LevelDesc* levels,
                     int nlev, uint32_t total_tiles, const uint32_t* perm, FieldMeta* meta,
                     cstream s);
void launch_bitlen(FieldMeta* meta, cstream s);
void launch_encode(const void* f, int dtype, const uint64_t dims[3], const LevelDesc* levels,
                   int nlev, uint32_t total_tiles, const uint32_t* perm, FieldMeta* meta,
                   uint32_t* planes, cstream s);
void launch_bitplane_encode(const void* q, const uint8_t* sign, uint64_t n, int B,
                            uint32_t* planes, cstream s);
void launch_bpd_encode(const uint32_t* q, const uint8_t* sign, uint64_t n, int design,
                       uint32_t* planes, cstream s);
void launch_bpd_decode(const uint32_t* planes, uint64_t n, int design, int k, uint32_t* q,
                       uint8_t* sign, cstream s);
void launch_bitplane_decode(const uint32_t* planes, uint64_t n, int B, int k, void* q,
                            uint8_t* sign, cstream s);

// lossless.cu
struct ChunkMap {
  const uint32_t* chunk_group;  // global chunk -> flat group index (l * ngroups + g)
  uint32_t total_chunks;
};
// group_hist (256 per group) and group_cost (per group) must start at zero
void launch_chunk_stats(const uint8_t* planes, FieldMeta* meta, ChunkMap cm, uint32_t* group_hist,
                        unsigned long long* group_cost, uint32_t* chunk_cost, cstream s);
// refactor: device-built lists of the Huffman and RLE chunks (lists holds
// 2 total_chunks entries, counts 2 zeroed words), and the coders over them
void launch_coder_lists(const FieldMeta* meta, ChunkMap cm, uint32_t* lists, uint32_t* counts,
                        cstream s);
void launch_huff_bits_list(const uint8_t* planes, const FieldMeta* meta, ChunkMap cm,
                           const uint8_t* lens, uint32_t* chunk_words, const uint32_t* lists,
                           const uint32_t* counts, cstream s);
void launch_huff_encode_list(const uint8_t* planes, const FieldMeta* meta, ChunkMap cm,
                             const uint8_t* lens, const uint32_t* chunk_out, uint8_t* slots,
                             const uint32_t* lists, const uint32_t* counts, cstream s);
void launch_rle_encode_list(const uint8_t* planes, const FieldMeta* meta, ChunkMap cm,
                            const uint32_t* chunk_out, uint8_t* slots, const uint32_t* lists,
                            const uint32_t* counts, cstream s);
void launch_decide(FieldMeta* meta, int ngroups_total, const uint32_t* group_hist,
                   const unsigned long long* group_cost, uint8_t* lens, uint64_t Ts,
                   uint32_t cr_num, uint32_t cr_den, int force, cstream s);
void launch_huff_bits(const uint8_t* planes, const FieldMeta* meta, ChunkMap cm, const uint8_t* lens,
                      uint32_t* chunk_words, cstream s);
void launch_group_offsets(FieldMeta* meta, int ngroups_total, const uint32_t* chunk_words,
                          const uint32_t* chunk_cost, uint32_t* chunk_out, cstream s);
void launch_huff_encode(const uint8_t* planes, const FieldMeta* meta, ChunkMap cm,
                        const uint8_t* lens, const uint32_t* chunk_out, uint8_t* slots, cstream s);
void launch_rle_encode(const uint8_t* planes, const FieldMeta* meta, ChunkMap cm,
                       const uint32_t* chunk_out, uint8_t* slots, cstream s);
void launch_headers(FieldMeta* meta, int ngroups_total, const uint8_t* lens,
                    const uint32_t* chunk_out, uint8_t* slots, cstream s);
void launch_decode(const uint8_t* slots, FieldMeta* meta, const RetrieveDev* rd,
                   uint32_t max_items, uint8_t* planes, cstream s);

// select.cu
// The groups used per level l <= l_end by a retrieval (l_end < 0: none given)
struct SmallSel {
  int32_t l_end;
  int32_t cur[HP_MAX_LEVELS];
};
void launch_sequence(FieldMeta* meta, cstream s);
// hs (may be null): a host selection of the small levels, checked against the
// device's (a mismatch sets the retrieval status to HPMDR_ERR_CORRUPT)
void launch_select(FieldMeta* meta, double tau, int tau_is_abs, RetrieveDev* rd, cstream s,
                   const SmallSel* hs = nullptr);
// k_select's choice for levels 0 .. l_end, computed on the host from its copy
// of the metadata, so that those levels can be recomposed beside k_select
void host_select_small(const FieldMeta& m, double tau, int tau_is_abs, int l_end, SmallSel* out);

// recompose.cu  (final_dtype: -1 = int64 level grid, 0 = float out, 1 = double out)
void launch_recompose_root(const uint32_t* planes, const FieldMeta* meta, const LevelDesc* L0,
                           int64_t* xroot, void* out, int dtype, cstream s);
void launch_convert_fixed(const int64_t* X, uint64_t n, int E_f, int dtype, void* out, cstream s);
void launch_recompose_copy(const LevelDesc* Lh, const LevelDesc& Lh_host, const int64_t* coarse,
                           void* dst, int final_dtype, const FieldMeta* meta, cstream s);
void launch_recompose_level(const uint32_t* planes, const FieldMeta* meta, const LevelDesc* Lh,
                            const LevelDesc& Lh_host, const uint32_t* perm, const int64_t* coarse,
                            void* dst, int B, int final_dtype, cstream s);
// root + levels 1..l_end (generic, small) in one CTA; levels_host: the host
// copy of the level descriptors
// hs (may be null): the groups per small level from host_select_small, used
// instead of the metadata's current selection (which k_select may be writing)
void launch_recompose_small(const uint32_t* planes, const FieldMeta* meta, const LevelDesc* levels,
                            const LevelDesc* levels_host, int l_end, int nlev, int64_t* xroot,
                            int64_t* xa, int64_t* xb, void* out, int dtype, cstream s,
                            const SmallSel* hs = nullptr);

// cells.cu (levels with g_x a multiple of 64; FP32, B = 32, or FP64, B = 64)
bool cell_path_ok(const LevelDesc& L, int B);
// est_done: the FP32 estimate of this level came with the statistics pass
void launch_cells_levelmax(const void* f, int dtype, const uint64_t dims[3], const LevelDesc* Ld,
                           const LevelDesc& Lh, FieldMeta* meta, cstream s, bool est_done = false);
// the field statistics and the finest level's FP32 estimate in one read of the
// field (FP32 fields whose finest level takes the cell kernels)
bool stats_cells_ok(int dtype, const LevelDesc& finest);
void launch_stats_cells(const float* f, const uint64_t dims[3], const LevelDesc* Ld,
                        const LevelDesc& Lh, FieldMeta* meta, cstream s);
void launch_cells_encode(const void* f, int dtype, const uint64_t dims[3], const LevelDesc* Ld,
                         const LevelDesc& Lh, FieldMeta* meta, uint32_t* planes, cstream s);
void launch_cells_recompose(const uint32_t* planes, const FieldMeta* meta, const LevelDesc* Ld,
                            const LevelDesc& Lh, const int64_t* coarse, void* dst, int final,
                            int B, cstream s);

// batched stage launchers (one launch covers every job).  unit0 tables live
// in device memory; `grid` is the persistent grid size.
void launch_b_init(const BatchJob* jobs, uint32_t njobs, cstream s);
void launch_b_stats(const BatchJob* jobs, const uint32_t* unit0, uint32_t njobs, uint32_t total,
                    uint32_t seg, int dtype, uint32_t grid, cstream s);
void launch_b_finalize(const BatchJob* jobs, uint32_t njobs, cstream s);
void launch_b_levelmax(const BatchJob* jobs, const uint32_t* unit0, uint32_t njobs, uint32_t total,
                       int dtype, uint32_t grid, cstream s);
void launch_b_bitlen(const BatchJob* jobs, uint32_t njobs, cstream s);
void launch_b_encode(const BatchJob* jobs, const uint32_t* unit0, uint32_t njobs, uint32_t total,
                     int dtype, uint32_t grid, cstream s);
void launch_b_cells_levelmax(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                             uint32_t nrefs, uint32_t total, uint32_t grid, int dtype, cstream s);
void launch_b_cells_encode(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                           uint32_t nrefs, uint32_t total, uint32_t grid, int dtype, cstream s);
void launch_b_cells_recompose(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                              uint32_t nrefs, uint32_t total, uint32_t grid, int dtype,
                              cstream s);
uint32_t cell_tiles(const LevelDesc& L);
void launch_b_chunk_stats(const BatchJob* jobs, const uint32_t* unit0, uint32_t njobs,
                          uint32_t total, uint32_t grid, cstream s);
void launch_b_decide(const BatchJob* jobs, const uint32_t* unit0, uint32_t njobs, uint32_t total,
                     uint64_t Ts, uint32_t cr_num, uint32_t cr_den, int force, uint32_t grid,
                     cstream s);
void launch_b_huff_bits(const BatchJob* jobs, const uint32_t* unit0, uint32_t njobs,
                        uint32_t total, uint32_t grid, cstream s);
void launch_b_group_offsets(const BatchJob* jobs, const uint32_t* unit0, uint32_t njobs,
                            uint32_t total, uint32_t grid, cstream s);
void launch_b_huff_encode(const BatchJob* jobs, const uint32_t* unit0, uint32_t njobs,
                          uint32_t total, uint32_t grid, cstream s);
void launch_b_rle_encode(const BatchJob* jobs, const uint32_t* unit0, uint32_t njobs,
                         uint32_t total, uint32_t grid, cstream s);
void launch_b_headers(const BatchJob* jobs, const uint32_t* unit0, uint32_t njobs, uint32_t total,
                      uint32_t grid, cstream s);
void launch_b_sequence(const BatchJob* jobs, uint32_t njobs, cstream s);
void launch_b_select(const BatchJob* jobs, uint32_t njobs, cstream s);
// unit0_out[j] = sum of rd->items of jobs before j (njobs + 1 entries)
void launch_b_items_prefix(const BatchJob* jobs, uint32_t njobs, uint32_t* unit0_out, cstream s);
void launch_b_decode(const BatchJob* jobs, const uint32_t* unit0_dev, uint32_t njobs,
                     uint32_t grid, cstream s);
void launch_b_recompose_small(const BatchJob* jobs, uint32_t njobs, int dtype, cstream s);
void launch_b_recompose_copy(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                             uint32_t nrefs, uint32_t total, int dtype, uint32_t grid, cstream s);
void launch_b_recompose_level(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                              uint32_t nrefs, uint32_t total, int dtype, uint32_t grid, cstream s);
void launch_b_gcells_levelmax(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                              uint32_t nrefs, uint32_t total, int dtype, uint32_t grid, cstream s);
void launch_b_gcells_encode(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                            uint32_t nrefs, uint32_t total, int dtype, uint32_t grid, cstream s);
void launch_b_gcells_recompose(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                               uint32_t nrefs, uint32_t total, int dtype, uint32_t grid,
                               cstream s);
void launch_b_pack(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                   uint32_t nrefs, uint32_t total, int B, uint32_t grid, cstream s);
void launch_b_unpack(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                     uint32_t nrefs, uint32_t total, int B, uint32_t grid, cstream s);
// contiguous copies of every job's FieldMeta and RetrieveDev (for one download)
void launch_b_gather(const BatchJob* jobs, uint32_t njobs, FieldMeta* metas, RetrieveDev* rds,
                     int32_t* statuses, cstream s);

// gcells.cu (any level grid with h >= 1, either precision): coefficients
// staged level-linear (q, sign), then Algorithm 1 by launch_bitplane_encode;
// on retrieval launch_level_unpack fills the staging buffer
void launch_gcells_levelmax(const void* f, int dtype, const uint64_t dims[3], const LevelDesc* Ld,
                            const LevelDesc& Lh, FieldMeta* meta, cstream s);
void launch_gcells_encode(const void* f, int dtype, const uint64_t dims[3], const LevelDesc* Ld,
                          const LevelDesc& Lh, FieldMeta* meta, void* q, uint8_t* sign,
                          cstream s);
void launch_gcells_recompose(const FieldMeta* meta, const LevelDesc* Ld, const LevelDesc& Lh,
                             int dtype, const void* q, const uint8_t* sign, const int64_t* coarse,
                             void* dst, int final, cstream s);
void launch_level_unpack(const uint32_t* planes, const FieldMeta* meta, const LevelDesc* Ld,
                         const LevelDesc& Lh, int B, void* q, uint8_t* sign, cstream s);

// qoi.cu
void launch_vmag_range(const float* vx, const float* vy, const float* vz, uint64_t N,
                       float* qrange /* device: [min, max] */, cstream s);
void launch_vmag(const float* vx, const float* vy, const float* vz, uint64_t N, float* out,
                 cstream s);
// total velocity V = vx^2 + vy^2 + vz^2 (FP64 evaluation, FP32 output)
void launch_vtotal_range(const float* vx, const float* vy, const float* vz, uint64_t N,
                         double* vrange /* device: [min, max] */, cstream s);
uint32_t vtotal_bound_blocks(uint64_t N);
// bytes of the scratch `best` of launch_vtotal_bound (8-byte aligned)
uint64_t vtotal_bound_scratch(uint64_t N);
// a 3-double slot inside that scratch for a caller's data error bounds
double* vtotal_bound_e(unsigned long long* best, uint64_t N);
// out = V_hat; best[0] = bits of the largest pointwise bound, best[1] = its
// first point (best holds vtotal_bound_scratch(N) bytes).  e: device
// addresses of the three data error bounds, read when the kernels run.
void launch_vtotal_bound(const float* vx, const float* vy, const float* vz, uint64_t N,
                         const double* const e[3], float* out, unsigned long long* best,
                         cstream s);

}  // namespace hp
