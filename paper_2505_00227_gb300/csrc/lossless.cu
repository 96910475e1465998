// Hybrid lossless coding of merged bitplane groups (Sec. 5): Huffman, RLE and
// direct copy, chosen per group by Algorithm 2 from light-weight size
// estimates (Sec. 5.2), plus the matching decoders used on retrieval.
//
// Formats (all little-endian, payload chunked by 16 KiB of input):
//   Huffman: u64 orig_len, u32 chunk_bytes, u32 nchunks, u8 len[256],
//            u32 word_off[nchunks+1], payload words; canonical codes in
//            (length, symbol) order, written MSB-first, each chunk starting on
//            a fresh 32-bit word.
//   RLE:     u64 orig_len, u32 chunk_bytes, u32 nchunks, u32 byte_off[nchunks+1],
//            payload of (byte, LEB128(run-1)) records; runs end at chunk ends.
//   DC:      the group bytes as they are (they stay in the plane buffer).
//
// GPU mapping: one CTA per 16 KiB chunk for statistics and encoding (chunk in
// shared memory), one CTA per group for the decision, one CTA of 512 threads
// per chunk for decoding (512 speculative Huffman segments; an RLE chunk is
// decoded by the CTA's first warp).  No inter-CTA waits anywhere.
#include "dev_common.cuh"

namespace hp {

__device__ __forceinline__ uint32_t huff_header_bytes(uint32_t nchunks) {
  return 8 + 4 + 4 + 256 + 4 * (nchunks + 1);
}
__device__ __forceinline__ uint32_t rle_header_bytes(uint32_t nchunks) {
  return 8 + 4 + 4 + 4 * (nchunks + 1);
}

struct ChunkRef {
  const GroupMeta* gm;
  uint32_t gi, cl, len;  // flat group index, chunk within group, bytes in chunk
  uint64_t start;        // byte offset of the chunk within the group
};

__device__ __forceinline__ ChunkRef chunk_ref(const FieldMeta* meta, const uint32_t* chunk_group,
                                              uint32_t c) {
  ChunkRef r;
  r.gi = chunk_group[c];
  const int ng = meta->ngroups;
  r.gm = &meta->grp[r.gi / ng][r.gi % ng];
  r.cl = c - r.gm->chunk0;
  r.start = (uint64_t)r.cl * HP_CHUNK;
  uint64_t rest = r.gm->S - r.start;
  r.len = (uint32_t)(rest < HP_CHUNK ? rest : HP_CHUNK);
  return r;
}

// load one chunk (16-byte aligned start) into shared memory: 128-bit loads for
// the bulk, bytes for a ragged tail
__device__ __forceinline__ void load_chunk(const uint8_t* __restrict__ src, uint32_t len,
                                           uint8_t* dst) {
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
  uint4* d4 = reinterpret_cast<uint4*>(dst);
  for (uint32_t i = threadIdx.x; i < len / 16; i += blockDim.x) d4[i] = __ldcs(s4 + i);
  for (uint32_t i = (len & ~15u) + threadIdx.x; i < len; i += blockDim.x) dst[i] = src[i];
}

// ------------------------------------------------- statistics per 16 KiB chunk
// byte histogram (for the Huffman estimate) and the exact RLE cost
// sum over runs of (1 + LEB128 length of run-1) = 2 runs + #(runs >= 129).
// Thread t owns bytes [64t, 64t+64) in registers: run starts are a 64-bit mask
// (a byte differing from its predecessor, the chunk's first byte always), and
// only a segment's last run can reach 129 bytes, so its length comes from the
// first run start of the following segments (a block-wide suffix minimum).
// Zero bytes are not counted one by one: the zero bin is the chunk's length
// less the other bins.  The histogram has four interleaved copies (bin v of copy
// c at word 4 v + c, lane l updating copy l & 3): lanes of different copies
// never share a bank, so a warp's atomic update needs fewer passes than with one
// copy per warp.  The work per byte is integer issue, so the inner loops keep
// it to a shift and a mask for the bin's byte offset.
__device__ __forceinline__ void chunk_stats_unit(const uint8_t* __restrict__ planes,
                                                     const FieldMeta* __restrict__ meta,
                                                     const uint32_t* __restrict__ chunk_group,
                                                     uint32_t* __restrict__ group_hist,
                                                     unsigned long long* __restrict__ group_cost,
                                                     uint32_t* __restrict__ chunk_cost,
    uint32_t c_unit) {
  __shared__ __align__(16) uint32_t hist[4 * 256];
  __shared__ uint32_t s_first[256], s_wmin[8];
  __shared__ uint8_t s_last[256];
  __shared__ uint32_t red[16];
  const uint32_t c = c_unit, t = threadIdx.x;
  const int lane = t & 31, w = t >> 5;
  if (meta->status) return;
  ChunkRef r = chunk_ref(meta, chunk_group, c);
  for (int i = t; i < 4 * 256; i += blockDim.x) hist[i] = 0;
  const uint32_t lo4 = 4u * (lane & 3);  // byte offset of this lane's copy: bin v at 16 v + lo4
  auto bump = [&](uint32_t off16, uint32_t n) {  // off16 = 16 v, v > 0
    atomicAdd(reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(hist) + (off16 | lo4)), n);
  };
  const uint8_t* src = planes + r.gm->plane_off + r.start;
  const uint32_t a = 64 * t, b = min(r.len, a + 64u), nb = b > a ? b - a : 0u;
  uint32_t wv[16];
  if (nb == 64) {
    const uint4* s4 = reinterpret_cast<const uint4*>(src + a);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint4 v = __ldcs(s4 + k);
      wv[4 * k] = v.x;
      wv[4 * k + 1] = v.y;
      wv[4 * k + 2] = v.z;
      wv[4 * k + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 16; k++) {
      uint32_t x = 0;
      for (int q = 0; q < 4; q++)
        if (4u * k + q < nb) x |= (uint32_t)src[a + 4 * k + q] << (8 * q);
      wv[k] = x;
    }
  }
  if (nb) {  // the segment's last byte (a select over the words keeps wv in registers)
    const uint32_t kl = (nb - 1) / 4;
    uint32_t lw = wv[15];
#pragma unroll
    for (int k = 0; k < 15; k++) lw = (uint32_t)k == kl ? wv[k] : lw;
    s_last[t] = (uint8_t)(lw >> (8 * ((nb - 1) % 4)));
  }
  __syncthreads();
  // run starts and histogram
  uint64_t mask = 0;
  if (nb == 64) {  // whole segment: a word at a time
    uint32_t pb = t > 0 ? s_last[t - 1] : 0u;
    uint32_t mlo = 0, mhi = 0;  // run starts of bytes 0..31 and 32..63
#pragma unroll
    for (int k = 0; k < 16; k++) {
      const uint32_t x = wv[k];
      if ((x | pb) == 0) continue;  // four zero bytes after a zero byte: no run starts
      const uint32_t d = x ^ ((x << 8) | pb);  // each byte against its predecessor
      const uint32_t nz = (((d & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | d) & 0x80808080u;
      // bits 7, 15, 23, 31 to bits 28..31 (the partial products never overlap)
      const uint32_t g = (nz * 0x204081u) >> 28;
      if (k < 8) mlo |= g << (4 * k);
      else mhi |= g << (4 * (k - 8));
      pb = x >> 24;
      if ((nz & 0x80808000u) == 0) {  // four equal bytes: one update
        if (x & 0xffu) bump((x << 4) & 0xff0u, 4u);
      } else {
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const uint32_t off = (q == 0 ? x << 4 : x >> (8 * q - 4)) & 0xff0u;
          if (off) bump(off, 1u);
        }
      }
    }
    mask = (uint64_t)mhi << 32 | mlo;
    if (t == 0) mask |= 1ull;  // the chunk's first byte starts a run
  } else {
    uint32_t prev = (t > 0 && nb) ? s_last[t - 1] : 0x100u;  // 0x100: the chunk start
#pragma unroll
    for (int k = 0; k < 16; k++) {
      const uint32_t x = wv[k];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const uint32_t idx = 4 * k + q;
        if (idx < nb) {
          const uint32_t v = (x >> (8 * q)) & 0xffu;
          if (v != prev) mask |= 1ull << idx;
          prev = v;
          if (v) bump(16u * v, 1u);
        }
      }
    }
  }
  // first run start of each segment, suffix minimum over the following segments
  const uint32_t INF = 0xffffffffu;
  uint32_t f = mask ? a + (uint32_t)(__ffsll((long long)mask) - 1) : INF;
  uint32_t sm = f;  // inclusive suffix min inside the warp
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_down_sync(HP_FULL, sm, d);
    if (lane + d < 32) sm = min(sm, o);
  }
  if (lane == 0) s_wmin[w] = sm;
  s_first[t] = sm;
  __syncthreads();
  uint32_t next;  // first run start after this segment (chunk end if none)
  {
    uint32_t nx = lane < 31 ? s_first[t + 1] : INF;
    for (int k = w + 1; k < 8; k++) nx = min(nx, s_wmin[k]);
    next = nx == INF ? r.len : nx;
  }
  uint32_t cost = 2u * (uint32_t)__popcll((long long)mask);
  if (mask) {
    const uint32_t last = a + 63u - (uint32_t)__clzll((long long)mask);
    if (next - last >= 129u) cost += 1;
  }
  __syncthreads();
  uint32_t nzb;  // the group's histogram is the sum over its chunks (integer atomics: exact)
  {
    const uint4 h = reinterpret_cast<const uint4*>(hist)[t];  // the four copies of bin t (0 for t = 0)
    nzb = h.x + h.y + h.z + h.w;
    if (nzb) atomicAdd(&group_hist[(size_t)r.gi * 256 + t], nzb);
  }
  for (int o = 16; o; o >>= 1) {
    cost += __shfl_xor_sync(HP_FULL, cost, o);
    nzb += __shfl_xor_sync(HP_FULL, nzb, o);
  }
  if (lane == 0) red[w] = cost, red[8 + w] = nzb;
  __syncthreads();
  if (t == 0) {
    uint32_t s = 0, nonzero = 0;
    for (int k = 0; k < 8; k++) s += red[k], nonzero += red[8 + k];
    if (r.len > nonzero) atomicAdd(&group_hist[(size_t)r.gi * 256], r.len - nonzero);  // zero bytes
    chunk_cost[c] = s;
    atomicAdd(&group_cost[r.gi], (unsigned long long)s);
  }
}

__global__ void __launch_bounds__(256) k_chunk_stats(const uint8_t* __restrict__ planes,
                                                     const FieldMeta* __restrict__ meta,
                                                     const uint32_t* __restrict__ chunk_group,
                                                     uint32_t* __restrict__ group_hist,
                                                     unsigned long long* __restrict__ group_cost,
                                                     uint32_t* __restrict__ chunk_cost) {
  hp::pdl_enter();
  chunk_stats_unit(planes, meta, chunk_group, group_hist, group_cost, chunk_cost, blockIdx.x);
}

void launch_chunk_stats(const uint8_t* planes, FieldMeta* meta, ChunkMap cm, uint32_t* group_hist,
                        unsigned long long* group_cost, uint32_t* chunk_cost, cstream s) {
  if (cm.total_chunks == 0) return;
  hp::note_launch(), hp::launch_pdl(k_chunk_stats, cm.total_chunks, 256, 0, s, planes, meta, cm.chunk_group,
                                                                   group_hist, group_cost,
                                                                   chunk_cost);
}

// -------------------------------------------- Algorithm 2 decision per group
// Huffman code lengths of the two-queue construction (leaves by (freq,
// symbol), a leaf wins a weight tie, internal nodes in creation order), capped
// at 16 by halving the counts and rebuilding.
__device__ void huffman_lengths_block(const uint64_t* f_in, uint8_t* len_out, uint64_t* f,
                                      int* sorted, uint64_t* w, int* parent, int* depth, int* flag) {
  const int t = threadIdx.x;  // 256 threads, t = symbol
  __shared__ int s_max;
  f[t] = f_in[t];
  __syncthreads();
  for (int round = 0; round < 64; round++) {
    // rank of symbol t among the nonzero symbols by (freq, symbol)
    int rank = 0, n = 0;
    uint64_t ft = f[t];
    for (int s = 0; s < 256; s++) {
      uint64_t fs = f[s];
      if (fs > 0) {
        n++;
        if (fs < ft || (fs == ft && s < t)) rank++;
      }
    }
    if (ft > 0) sorted[rank] = t;
    len_out[t] = 0;
    if (t == 0) s_max = 0;
    __syncthreads();
    if (n > 1) {
      // The two-queue merge (leaves in (freq, symbol) order, internal nodes in
      // creation order, a leaf first on equal weights) consumes the items in the
      // order of the stable merge M of the leaves and the internal nodes, two per
      // step: internal j = M[2j] + M[2j+1].  That is a fixed point in the
      // internal weights, found here in parallel instead of by one thread.
      // Started from +inf, the iterates stay sorted (pair sums of a sorted
      // sequence) and no smaller than the true weights, and after r rounds the
      // first r internal weights are exact: the loop ends by round n at the
      // latest, with the merge positions of the exact weights.
      __shared__ uint64_t s_m[512];
      const uint64_t INF = ~0ull;
      uint64_t* L = w;        // leaves w[0, n)
      uint64_t* I = w + 256;  // internal nodes w[256, 256 + n - 1)
      if (t < n) L[t] = f[sorted[t]];
      if (t < n - 1) I[t] = INF;
      __syncthreads();
      int pl = 0, pi = 0;  // merge positions of leaf t and internal node t
      for (int r = 0; r < n; r++) {
        if (t < n) {  // leaf t follows t leaves and the internal nodes lighter than it
          const uint64_t x = L[t];
          int lo = 0, hi = n - 1;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (I[mid] < x) lo = mid + 1;
            else hi = mid;
          }
          pl = t + lo;
          s_m[pl] = x;
        }
        if (t < n - 1) {  // internal t follows t internal nodes and the leaves not heavier
          const uint64_t y = I[t];
          int lo = 0, hi = n;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (L[mid] <= y) lo = mid + 1;
            else hi = mid;
          }
          pi = t + lo;
          s_m[pi] = y;
        }
        __syncthreads();
        bool changed = false;
        if (t < n - 1) {
          const uint64_t a = s_m[2 * t], b = s_m[2 * t + 1];
          const uint64_t v = (a == INF || b == INF) ? INF : a + b;
          changed = v != I[t];
          I[t] = v;  // read only by thread t until the barrier below
        }
        if (!__syncthreads_or(changed ? 1 : 0)) break;
      }
      // node ids: leaf i = i, internal node j = n + j; the item at merge
      // position p hangs under internal node p / 2; the last one is the root
      if (t < n) parent[t] = n + (pl >> 1);
      if (t < n - 1) parent[n + t] = t == n - 2 ? n + t : n + (pi >> 1);
      __syncthreads();
      // depths by pointer jumping: d(v) accumulates along doubling ancestor links
      const int nodes = 2 * n - 1;
      for (int v = t; v < nodes; v += blockDim.x) depth[v] = v == nodes - 1 ? 0 : 1;
      __syncthreads();
      for (int it = 0; it < 9; it++) {  // depth < 256 <= 2^9
        int nd[2], na[2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
          const int v = t + u * 256;
          if (v < nodes) {
            const int a = parent[v];
            nd[u] = depth[v] + depth[a];
            na[u] = parent[a];
          }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 2; u++) {
          const int v = t + u * 256;
          if (v < nodes) {
            depth[v] = nd[u];
            parent[v] = na[u];
          }
        }
        __syncthreads();
      }
      if (t < n) {
        len_out[sorted[t]] = (uint8_t)depth[t];
        atomicMax(&s_max, depth[t]);
      }
    } else if (n == 1 && t == 0) {
      len_out[sorted[0]] = 1;
      s_max = 1;
    }
    __syncthreads();
    if (t == 0) *flag = s_max > 16;
    __syncthreads();
    if (!*flag) break;
    if (f[t] > 0) f[t] = (f[t] + 1) >> 1;
    __syncthreads();
  }
}

__device__ __forceinline__ void decide_unit(FieldMeta* meta, const uint32_t* __restrict__ group_hist,
                                                const unsigned long long* __restrict__ group_cost,
                                                uint8_t* __restrict__ lens, uint64_t Ts,
                                                uint32_t cr_num, uint32_t cr_den, int force,
    uint32_t g_unit) {
  __shared__ uint64_t hist[256], f[256], w[512];
  __shared__ int sorted[256], parent[512], depth[512], flag;
  __shared__ uint8_t len[256];
  __shared__ uint64_t red[8];
  if (meta->status) return;
  const uint32_t gi = g_unit;
  const int ng = meta->ngroups;
  GroupMeta* gm = &meta->grp[gi / ng][gi % ng];
  const int t = threadIdx.x;
  hist[t] = group_hist[(size_t)gi * 256 + t];
  if (t == 0) red[0] = group_cost[gi];
  __syncthreads();
  huffman_lengths_block(hist, len, f, sorted, w, parent, depth, &flag);
  __syncthreads();
  uint64_t bits = hist[t] * (uint64_t)len[t];
  bits = warp_sum_u64(bits);
  __shared__ uint64_t redb[8];
  if ((t & 31) == 0) redb[t >> 5] = bits;
  lens[(size_t)gi * 256 + t] = len[t];
  __syncthreads();
  if (t == 0) {
    uint64_t tb = 0, tc = red[0];
    for (int k = 0; k < 8; k++) tb += redb[k];
    const uint64_t S = gm->S;
    const uint32_t nc = gm->nchunks;
    uint64_t est_H = huff_header_bytes(nc) + (tb + 7) / 8 + 4ull * nc;
    uint64_t est_R = rle_header_bytes(nc) + tc;
    gm->est_H = est_H;
    gm->est_R = est_R;
    int m = 0;  // DC
    if (S > Ts) {
      unsigned __int128 lhs = (unsigned __int128)S * cr_den;
      if (lhs > (unsigned __int128)cr_num * est_H) m = 1;       // Huffman
      else if (lhs > (unsigned __int128)cr_num * est_R) m = 2;  // RLE
    }
    if (force >= 0) m = force;  // stage entry point: caller-chosen method
    gm->method = m;
    gm->stored_len = S;  // final for DC; set by the offsets pass otherwise
  }
}

__global__ void __launch_bounds__(256) k_decide(FieldMeta* meta, const uint32_t* __restrict__ group_hist,
                                                const unsigned long long* __restrict__ group_cost,
                                                uint8_t* __restrict__ lens, uint64_t Ts,
                                                uint32_t cr_num, uint32_t cr_den, int force) {
  hp::pdl_enter();
  decide_unit(meta, group_hist, group_cost, lens, Ts, cr_num, cr_den, force, blockIdx.x);
}

void launch_decide(FieldMeta* meta, int ngroups_total, const uint32_t* group_hist,
                   const unsigned long long* group_cost, uint8_t* lens, uint64_t Ts,
                   uint32_t cr_num, uint32_t cr_den, int force, cstream s) {
  hp::note_launch(), hp::launch_pdl(k_decide, ngroups_total, 256, 0, s, meta, group_hist, group_cost, lens, Ts,
                                                            cr_num, cr_den, force);
}

// block-wide exclusive prefix sum (any thread count that is a multiple of 32,
// up to 1024); returns the inclusive total too
__device__ __forceinline__ uint32_t block_exscan(uint32_t v, uint32_t* scratch, uint32_t& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(HP_FULL, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) scratch[w] = x;
  __syncthreads();
  uint32_t base = 0, all = 0;
  for (int k = 0; k < nw; k++) {
    if (k < w) base += scratch[k];
    all += scratch[k];
  }
  __syncthreads();
  total = all;
  return base + x - v;
}

// --------------------------------------------------- canonical Huffman codes
// code[t] for the canonical code of lengths len[] ((length, symbol) order),
// 256 threads: a symbol's rank among the symbols of its length is the count in
// earlier warps (per-warp length counts) plus the earlier lanes of its own
// warp holding the same length (a warp match)
__device__ void canonical_codes_block(const uint8_t* len, uint32_t* code, uint32_t* first) {
  __shared__ uint32_t wcnt[8][17];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  if (t < 8 * 17) (&wcnt[0][0])[t] = 0;
  __syncthreads();
  const uint32_t L = len[t];
  const unsigned same = __match_any_sync(HP_FULL, L);
  if ((int)(__ffs(same) - 1) == lane) wcnt[w][L] = __popc(same);  // one writer per length
  __syncthreads();
  if (t == 0) {
    uint32_t c = 0;
    for (int l = 1; l <= 16; l++) {
      first[l] = c;
      uint32_t n = 0;
      for (int k = 0; k < 8; k++) n += wcnt[k][l];
      c = (c + n) << 1;
    }
  }
  __syncthreads();
  if (L) {
    uint32_t r = __popc(same & ((1u << lane) - 1u));
    for (int k = 0; k < w; k++) r += wcnt[k][L];
    code[t] = first[L] + r;
  } else {
    code[t] = 0;
  }
  __syncthreads();
}

// --------------------------------------------------- Huffman: bits per chunk
__device__ __forceinline__ void huff_bits_unit(const uint8_t* __restrict__ planes,
                                                   const FieldMeta* __restrict__ meta,
                                                   const uint32_t* __restrict__ chunk_group,
                                                   const uint8_t* __restrict__ lens,
                                                   uint32_t* __restrict__ chunk_words,
    uint32_t c_unit) {
  __shared__ uint8_t len[256];
  __shared__ uint32_t red[8];
  if (meta->status) return;
  ChunkRef r = chunk_ref(meta, chunk_group, c_unit);
  if (r.gm->method != 1) return;
  len[threadIdx.x] = lens[(size_t)r.gi * 256 + threadIdx.x];
  __syncthreads();
  const uint8_t* src = planes + r.gm->plane_off + r.start;
  uint32_t bits = 0;
  const uint32_t z4 = 4u * len[0];  // a word of four zero bytes
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
  for (uint32_t i = threadIdx.x; i < r.len / 16; i += blockDim.x) {
    uint4 v = __ldcs(s4 + i);
    uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; k++) {
      if (wv[k] == 0) {
        bits += z4;
        continue;
      }
#pragma unroll
      for (int b = 0; b < 4; b++) bits += len[(wv[k] >> (8 * b)) & 0xffu];
    }
  }
  for (uint32_t i = (r.len & ~15u) + threadIdx.x; i < r.len; i += blockDim.x) bits += len[src[i]];
  for (int o = 16; o; o >>= 1) bits += __shfl_xor_sync(HP_FULL, bits, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = bits;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int k = 0; k < 8; k++) s += red[k];
    chunk_words[c_unit] = (s + 31) / 32;
  }
}

__global__ void __launch_bounds__(256) k_huff_bits(const uint8_t* __restrict__ planes,
                                                   const FieldMeta* __restrict__ meta,
                                                   const uint32_t* __restrict__ chunk_group,
                                                   const uint8_t* __restrict__ lens,
                                                   uint32_t* __restrict__ chunk_words) {
  hp::pdl_enter();
  huff_bits_unit(planes, meta, chunk_group, lens, chunk_words, blockIdx.x);
}

void launch_huff_bits(const uint8_t* planes, const FieldMeta* meta, ChunkMap cm, const uint8_t* lens,
                      uint32_t* chunk_words, cstream s) {
  if (cm.total_chunks == 0) return;
  hp::note_launch(), hp::launch_pdl(k_huff_bits, cm.total_chunks, 256, 0, s, planes, meta,
                                    cm.chunk_group, lens, chunk_words);
}

// ------------------------------------------- coder work lists (refactor)
// The chunks of the Huffman groups (lists[0 ..)) and of the RLE groups
// (lists[tc ..)), appended in any order; counts[0], counts[1] start at zero.
// The coder kernels then run persistent CTAs over their own list instead of a
// CTA per chunk of the field (most chunks belong to direct-copy groups).
__global__ void k_coder_lists(const FieldMeta* __restrict__ meta,
                              const uint32_t* __restrict__ chunk_group, uint32_t tc,
                              uint32_t* __restrict__ lists, uint32_t* __restrict__ counts) {
  hp::pdl_enter();
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (meta->status) return;
  int m = 0;
  if (c < tc) {
    const uint32_t gi = chunk_group[c];
    const int ng = meta->ngroups;
    m = meta->grp[gi / ng][gi % ng].method;
  }
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 1; k <= 2; k++) {  // one atomic per warp and method
    const unsigned hit = __ballot_sync(HP_FULL, m == k);
    if (!hit) continue;
    uint32_t base = 0;
    if (lane == __ffs(hit) - 1) base = atomicAdd(&counts[k - 1], (uint32_t)__popc(hit));
    base = __shfl_sync(HP_FULL, base, __ffs(hit) - 1);
    if (m == k) lists[(k - 1) * (size_t)tc + base + __popc(hit & ((1u << lane) - 1u))] = c;
  }
}

void launch_coder_lists(const FieldMeta* meta, ChunkMap cm, uint32_t* lists, uint32_t* counts,
                        cstream s) {
  if (cm.total_chunks == 0) return;
  hp::note_launch(), hp::launch_pdl(k_coder_lists, (cm.total_chunks + 255) / 256, 256, 0, s, meta,
                                    cm.chunk_group, cm.total_chunks, lists, counts);
}

__global__ void __launch_bounds__(256) k_huff_bits_list(const uint8_t* __restrict__ planes,
                                                        const FieldMeta* __restrict__ meta,
                                                        const uint32_t* __restrict__ chunk_group,
                                                        const uint8_t* __restrict__ lens,
                                                        uint32_t* __restrict__ chunk_words,
                                                        const uint32_t* __restrict__ list,
                                                        const uint32_t* __restrict__ count) {
  hp::pdl_enter();
  const uint32_t n = *count;
  for (uint32_t e = blockIdx.x; e < n; e += gridDim.x) {
    huff_bits_unit(planes, meta, chunk_group, lens, chunk_words, list[e]);
    __syncthreads();
  }
}

static uint32_t coder_grid(uint32_t total, int per_sm) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint32_t cap = (uint32_t)(sms * per_sm);
  return total < cap ? (total ? total : 1u) : cap;
}

void launch_huff_bits_list(const uint8_t* planes, const FieldMeta* meta, ChunkMap cm,
                           const uint8_t* lens, uint32_t* chunk_words, const uint32_t* lists,
                           const uint32_t* counts, cstream s) {
  if (cm.total_chunks == 0) return;
  hp::note_launch(), hp::launch_pdl(k_huff_bits_list, coder_grid(cm.total_chunks, 8), 256, 0, s,
                                    planes, meta, cm.chunk_group, lens, chunk_words, lists, counts);
}

// ------------------------------------ per-group chunk output offsets (scan)
// Huffman: word offset of each chunk in the payload; RLE: byte offset.
__device__ __forceinline__ void group_offsets_unit(FieldMeta* meta,
                                                       const uint32_t* __restrict__ chunk_words,
                                                       const uint32_t* __restrict__ chunk_cost,
                                                       uint32_t* __restrict__ chunk_out,
    uint32_t g_unit) {
  __shared__ uint64_t part[256];
  if (meta->status) return;
  const uint32_t gi = g_unit;
  const int ng = meta->ngroups;
  GroupMeta* gm = &meta->grp[gi / ng][gi % ng];
  const int m = gm->method;
  if (m == 0) return;
  const uint32_t* src = (m == 1 ? chunk_words : chunk_cost) + gm->chunk0;
  const uint32_t nc = gm->nchunks, t = threadIdx.x;
  const uint32_t per = (nc + 255) / 256, a = t * per, b = min(nc, a + per);
  uint64_t s = 0;
  for (uint32_t c = a; c < b; c++) s += src[c];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    uint64_t run = 0;
    for (int k = 0; k < 256; k++) {
      uint64_t v = part[k];
      part[k] = run;
      run += v;
    }
    uint64_t hdr = m == 1 ? huff_header_bytes(nc) : rle_header_bytes(nc);
    uint64_t total = hdr + (m == 1 ? 4 * run : run);
    gm->stored_len = total;
    if (total > gm->cap) atomicExch(&meta->status, -4);  // cannot happen for T_cr >= 1
  }
  __syncthreads();
  uint64_t o = part[t];
  for (uint32_t c = a; c < b; c++) {
    chunk_out[gm->chunk0 + c] = (uint32_t)o;
    o += src[c];
  }
}

__global__ void __launch_bounds__(256) k_group_offsets(FieldMeta* meta,
                                                       const uint32_t* __restrict__ chunk_words,
                                                       const uint32_t* __restrict__ chunk_cost,
                                                       uint32_t* __restrict__ chunk_out) {
  hp::pdl_enter();
  group_offsets_unit(meta, chunk_words, chunk_cost, chunk_out, blockIdx.x);
}

void launch_group_offsets(FieldMeta* meta, int ngroups_total, const uint32_t* chunk_words,
                          const uint32_t* chunk_cost, uint32_t* chunk_out, cstream s) {
  hp::note_launch(), hp::launch_pdl(k_group_offsets, ngroups_total, 256, 0, s, meta, chunk_words,
                                    chunk_cost, chunk_out);
}

// -------------------------------------------------------- Huffman: encode
// Thread t codes bytes [64 t, 64 t + 64) of the chunk: its bit offset comes
// from a block scan of the code lengths, its bits are packed in a 64-bit
// register and written a word at a time; only its first and last words can be
// shared with a neighbour, and those are merged with atomicOr.
__device__ __forceinline__ void huff_encode_unit(const uint8_t* __restrict__ planes,
                                                     const FieldMeta* __restrict__ meta,
                                                     const uint32_t* __restrict__ chunk_group,
                                                     const uint8_t* __restrict__ lens,
                                                     const uint32_t* __restrict__ chunk_out,
                                                     uint8_t* __restrict__ slots,
    uint32_t c_unit) {
  __shared__ uint8_t len[256];
  __shared__ uint32_t code[256], first[17];
  __shared__ uint32_t outw[HP_CHUNK * 16 / 32];  // worst case: 16 bits per byte
  __shared__ uint32_t scratch[8];
  if (meta->status) return;
  ChunkRef r = chunk_ref(meta, chunk_group, c_unit);
  if (r.gm->method != 1) return;
  const int t = threadIdx.x;
  len[t] = lens[(size_t)r.gi * 256 + t];
  for (int i = t; i < HP_CHUNK * 16 / 32; i += 256) outw[i] = 0;
  __syncthreads();
  canonical_codes_block(len, code, first);
  const uint8_t* src = planes + r.gm->plane_off + r.start;
  const uint32_t a = t * 64u, nb = r.len > a ? min(r.len - a, 64u) : 0u;
  uint32_t wv[16];
  if (nb == 64) {  // cached loads: the code pass below reads the segment again
    const uint4* s4 = reinterpret_cast<const uint4*>(src + a);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint4 v = __ldg(s4 + k);
      wv[4 * k] = v.x;
      wv[4 * k + 1] = v.y;
      wv[4 * k + 2] = v.z;
      wv[4 * k + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 16; k++) {
      uint32_t x = 0;
      for (int q = 0; q < 4; q++)
        if (4u * k + q < nb) x |= (uint32_t)src[a + 4 * k + q] << (8 * q);
      wv[k] = x;
    }
  }
  // a word of four zero bytes (the common case in the sparse planes Huffman
  // wins on) appends code[0] four times in one step when it has <= 8 bits
  const uint32_t L0 = len[0];
  const bool zfast = L0 > 0 && L0 <= 8;
  const uint32_t c0 = code[0], z4len = 4 * L0;
  const uint32_t z4 = zfast ? (((c0 << L0 | c0) << L0 | c0) << L0 | c0) : 0u;
  uint32_t bits = 0;
#pragma unroll
  for (int k = 0; k < 16; k++) {
    if (zfast && wv[k] == 0 && 4u * k + 3 < nb) {
      bits += z4len;
      continue;
    }
#pragma unroll
    for (int q = 0; q < 4; q++)
      if (4u * k + q < nb) bits += len[(wv[k] >> (8 * q)) & 0xffu];
  }
  uint32_t total;
  const uint32_t pos = block_exscan(bits, scratch, total);
  uint64_t acc = 0;  // pending bits, MSB-aligned
  int nacc = (int)(pos & 31);
  uint32_t wd = pos >> 5;
  bool shared_word = true;  // the first word may hold the previous thread's bits
  // append L <= 32 bits of value v (nacc < 32 before, so < 64 after)
  auto put = [&](uint32_t v, int L) {
    acc |= (uint64_t)v << (64 - nacc - L);
    nacc += L;
    if (nacc >= 32) {
      const uint32_t hi = (uint32_t)(acc >> 32);
      if (shared_word) atomicOr(&outw[wd], hi);
      else outw[wd] = hi;
      shared_word = false;
      acc <<= 32;
      nacc -= 32;
      wd++;
    }
  };
  if (nb == 64) {
    // a whole segment: four 16-byte words per iteration, re-read from L1, so the
    // appends are not unrolled 64 times (the unrolled form missed the
    // instruction cache)
    const uint4* s4 = reinterpret_cast<const uint4*>(src + a);
#pragma unroll 1
    for (int j = 0; j < 4; j++) {
      const uint4 v = __ldg(s4 + j);
      const uint32_t ws[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int u = 0; u < 4; u++) {
        if (zfast && ws[u] == 0) {
          put(z4, (int)z4len);
          continue;
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const uint32_t sym = (ws[u] >> (8 * q)) & 0xffu;
          put(code[sym], (int)len[sym]);
        }
      }
    }
  } else {  // the ragged end of a group: bytes re-read one by one, up to nb
#pragma unroll 1
    for (uint32_t b = 0; b < nb; b++) {
      const uint32_t sym = src[a + b];
      put(code[sym], (int)len[sym]);
    }
  }
  if (nacc > 0 && bits > 0) atomicOr(&outw[wd], (uint32_t)(acc >> 32));  // shared with the next
  __syncthreads();
  const uint32_t nwords = (total + 31) / 32;
  uint32_t* dst = reinterpret_cast<uint32_t*>(slots + r.gm->slot_off +
                                              huff_header_bytes(r.gm->nchunks)) +
                  chunk_out[c_unit];
  for (uint32_t i = t; i < nwords; i += 256) dst[i] = outw[i];
}

__global__ void __launch_bounds__(256) k_huff_encode(const uint8_t* __restrict__ planes,
                                                     const FieldMeta* __restrict__ meta,
                                                     const uint32_t* __restrict__ chunk_group,
                                                     const uint8_t* __restrict__ lens,
                                                     const uint32_t* __restrict__ chunk_out,
                                                     uint8_t* __restrict__ slots) {
  hp::pdl_enter();
  huff_encode_unit(planes, meta, chunk_group, lens, chunk_out, slots, blockIdx.x);
}

__global__ void __launch_bounds__(256, 4) k_huff_encode_list(const uint8_t* __restrict__ planes,
                                                          const FieldMeta* __restrict__ meta,
                                                          const uint32_t* __restrict__ chunk_group,
                                                          const uint8_t* __restrict__ lens,
                                                          const uint32_t* __restrict__ chunk_out,
                                                          uint8_t* __restrict__ slots,
                                                          const uint32_t* __restrict__ list,
                                                          const uint32_t* __restrict__ count) {
  hp::pdl_enter();
  const uint32_t n = *count;
  for (uint32_t e = blockIdx.x; e < n; e += gridDim.x) {
    huff_encode_unit(planes, meta, chunk_group, lens, chunk_out, slots, list[e]);
    __syncthreads();
  }
}

void launch_huff_encode_list(const uint8_t* planes, const FieldMeta* meta, ChunkMap cm,
                             const uint8_t* lens, const uint32_t* chunk_out, uint8_t* slots,
                             const uint32_t* lists, const uint32_t* counts, cstream s) {
  if (cm.total_chunks == 0) return;
  hp::note_launch(), hp::launch_pdl(k_huff_encode_list, coder_grid(cm.total_chunks, 4), 256, 0, s,
                                    planes, meta, cm.chunk_group, lens, chunk_out, slots, lists,
                                    counts);
}

void launch_huff_encode(const uint8_t* planes, const FieldMeta* meta, ChunkMap cm,
                        const uint8_t* lens, const uint32_t* chunk_out, uint8_t* slots, cstream s) {
  if (cm.total_chunks == 0) return;
  hp::note_launch(), hp::launch_pdl(k_huff_encode, cm.total_chunks, 256, 0, s, planes, meta, cm.chunk_group, lens, chunk_out,
                                                slots);
}

// ------------------------------------------------------------ RLE: encode
__device__ __forceinline__ void rle_encode_unit(const uint8_t* __restrict__ planes,
                                                    const FieldMeta* __restrict__ meta,
                                                    const uint32_t* __restrict__ chunk_group,
                                                    const uint32_t* __restrict__ chunk_out,
                                                    uint8_t* __restrict__ slots,
    uint32_t c_unit) {
  __shared__ __align__(16) uint8_t buf[HP_CHUNK];
  __shared__ uint32_t scan[256];
  if (meta->status) return;
  ChunkRef r = chunk_ref(meta, chunk_group, c_unit);
  if (r.gm->method != 2) return;
  const int t = threadIdx.x;
  load_chunk(planes + r.gm->plane_off + r.start, r.len, buf);
  __syncthreads();
  const uint32_t a = t * 64u, b = min(r.len, a + 64u);
  uint32_t cost = 0;
  for (uint32_t i = a; i < b; i++) {
    if (i == 0 || buf[i - 1] != buf[i]) {
      uint32_t k = 1;
      while (i + k < r.len && buf[i + k] == buf[i]) k++;
      cost += 2 + (k > 128 ? 1u : 0u);
    }
  }
  scan[t] = cost;
  __syncthreads();
  if (t == 0) {
    uint32_t run = 0;
    for (int k = 0; k < 256; k++) {
      uint32_t v = scan[k];
      scan[k] = run;
      run += v;
    }
  }
  __syncthreads();
  uint8_t* dst = slots + r.gm->slot_off + rle_header_bytes(r.gm->nchunks) + chunk_out[c_unit] +
                 scan[t];
  uint32_t o = 0;
  for (uint32_t i = a; i < b; i++) {
    if (i == 0 || buf[i - 1] != buf[i]) {
      uint32_t k = 1;
      while (i + k < r.len && buf[i + k] == buf[i]) k++;
      dst[o++] = buf[i];
      uint32_t x = k - 1;
      while (x >= 128) {
        dst[o++] = (uint8_t)((x & 127u) | 128u);
        x >>= 7;
      }
      dst[o++] = (uint8_t)x;
    }
  }
}

__global__ void __launch_bounds__(256) k_rle_encode(const uint8_t* __restrict__ planes,
                                                    const FieldMeta* __restrict__ meta,
                                                    const uint32_t* __restrict__ chunk_group,
                                                    const uint32_t* __restrict__ chunk_out,
                                                    uint8_t* __restrict__ slots) {
  hp::pdl_enter();
  rle_encode_unit(planes, meta, chunk_group, chunk_out, slots, blockIdx.x);
}

__global__ void __launch_bounds__(256) k_rle_encode_list(const uint8_t* __restrict__ planes,
                                                         const FieldMeta* __restrict__ meta,
                                                         const uint32_t* __restrict__ chunk_group,
                                                         const uint32_t* __restrict__ chunk_out,
                                                         uint8_t* __restrict__ slots,
                                                         const uint32_t* __restrict__ list,
                                                         const uint32_t* __restrict__ count) {
  hp::pdl_enter();
  const uint32_t n = *count;
  for (uint32_t e = blockIdx.x; e < n; e += gridDim.x) {
    rle_encode_unit(planes, meta, chunk_group, chunk_out, slots, list[e]);
    __syncthreads();
  }
}

void launch_rle_encode_list(const uint8_t* planes, const FieldMeta* meta, ChunkMap cm,
                            const uint32_t* chunk_out, uint8_t* slots, const uint32_t* lists,
                            const uint32_t* counts, cstream s) {
  if (cm.total_chunks == 0) return;
  hp::note_launch(), hp::launch_pdl(k_rle_encode_list, coder_grid(cm.total_chunks, 4), 256, 0, s,
                                    planes, meta, cm.chunk_group, chunk_out, slots,
                                    lists + cm.total_chunks, counts + 1);
}

void launch_rle_encode(const uint8_t* planes, const FieldMeta* meta, ChunkMap cm,
                       const uint32_t* chunk_out, uint8_t* slots, cstream s) {
  if (cm.total_chunks == 0) return;
  hp::note_launch(), hp::launch_pdl(k_rle_encode, cm.total_chunks, 256, 0, s, planes, meta,
                                    cm.chunk_group, chunk_out, slots);
}

// ---------------------------------------------------------- group headers
__device__ __forceinline__ void headers_unit(const FieldMeta* __restrict__ meta,
                                                 const uint8_t* __restrict__ lens,
                                                 const uint32_t* __restrict__ chunk_out,
                                                 uint8_t* __restrict__ slots,
    uint32_t g_unit) {
  if (meta->status) return;
  const uint32_t gi = g_unit;
  const int ng = meta->ngroups;
  const GroupMeta* gm = &meta->grp[gi / ng][gi % ng];
  const int m = gm->method;
  if (m == 0) return;
  uint8_t* h = slots + gm->slot_off;
  const uint32_t nc = gm->nchunks, t = threadIdx.x;
  if (t == 0) {
    *reinterpret_cast<uint64_t*>(h) = gm->S;
    *reinterpret_cast<uint32_t*>(h + 8) = HP_CHUNK;
    *reinterpret_cast<uint32_t*>(h + 12) = nc;
  }
  uint32_t* offs;
  uint32_t endv;
  if (m == 1) {
    h[16 + t] = lens[(size_t)gi * 256 + t];
    offs = reinterpret_cast<uint32_t*>(h + 272);
    endv = (uint32_t)((gm->stored_len - huff_header_bytes(nc)) / 4);
  } else {
    offs = reinterpret_cast<uint32_t*>(h + 16);
    endv = (uint32_t)(gm->stored_len - rle_header_bytes(nc));
  }
  for (uint32_t c = t; c < nc; c += 256) offs[c] = chunk_out[gm->chunk0 + c];
  if (t == 0) offs[nc] = endv;
}

__global__ void __launch_bounds__(256) k_headers(const FieldMeta* __restrict__ meta,
                                                 const uint8_t* __restrict__ lens,
                                                 const uint32_t* __restrict__ chunk_out,
                                                 uint8_t* __restrict__ slots) {
  hp::pdl_enter();
  headers_unit(meta, lens, chunk_out, slots, blockIdx.x);
}

void launch_headers(FieldMeta* meta, int ngroups_total, const uint8_t* lens,
                    const uint32_t* chunk_out, uint8_t* slots, cstream s) {
  hp::note_launch(), hp::launch_pdl(k_headers, ngroups_total, 256, 0, s, meta, lens, chunk_out,
                                    slots);
}

// ================================================================ decoding
// One CTA of HP_DEC_THREADS threads per queued chunk (a Huffman chunk takes
// all of them, an RLE chunk the first warp).  Every read of the stored
// bytes is checked against the group's stored length; a failed check sets
// status CORRUPT and abandons the chunk (no trap).
__device__ __forceinline__ void set_corrupt(FieldMeta* meta) { atomicExch(&meta->status, -4); }

// Huffman decoding of one chunk by one CTA, self-synchronizing:
//  1. tables, built by all threads: canonical first code / count / sorted
//     symbols per length (lengths counted per warp with warp matches, ranks
//     among equal lengths from those counts) and a 10-bit lookup table for
//     short codes; a CTA keeps a group's tables across consecutive chunks;
//  2. the chunk's bits are cut into HP_DEC_THREADS segments whose starts lie on
//     the lattice of the gcd of the code lengths; thread i decodes from the
//     start of its segment (maybe mid-codeword) to the first codeword start at
//     or beyond the next segment, marking every start it visits in a bitmap
//     of the chunk's bits (runs of the one-bit code are taken up to 32
//     codewords at a time);
//  3. each thread's parse then continues past its segment until it lands on a
//     start marked by a later segment (from there both parses agree: Huffman
//     codes resynchronize) or runs off the data: its join point;
//  4. the true parse is segment 0's and hands over at each join to the segment
//     holding it.  When every segment joins the next one the emit ranges
//     follow at once; otherwise the chain of hand-overs from segment 0 is found
//     by pointer doubling.  Each chain segment counts its codewords from its
//     true start through its join, a prefix sum gives the output offsets, and
//     each chain segment decodes its span again, writing the bytes.
// The bitmap covers the longest possible chunk (16384 codes of 16 bits); a
// chunk claiming more bits is decoded by one thread and then fails its checks.
// All reads stay inside the chunk's words; an invalid code or a wrong symbol
// count marks the data corrupt.
#define HP_DEC_THREADS 512  // threads per decoded chunk: one speculative segment each
#define HP_DEC_SYMS ((256 + HP_DEC_THREADS - 1) / HP_DEC_THREADS)  // symbols per thread (tables)
#define HP_LUT_BITS 10
#define HP_MAP_WORDS 8192  // bitmap of 262144 bit positions per chunk: 16 bits x 16384 symbols

struct HuffTables {
  uint16_t lut[1 << HP_LUT_BITS];  // (len << 8) | symbol for codes of <= 10 bits, 0 otherwise
  uint32_t first[17];
  uint32_t count[17];
  uint32_t index[17];
  uint32_t fill[17];
  uint8_t sorted[256];
  uint32_t map[HP_MAP_WORDS];      // codeword starts of the speculative decodings
};

struct BitReader {
  const uint32_t* w;
  uint32_t nwords, wi;
  uint64_t buf;
  int nb;
  __device__ __forceinline__ uint32_t load(uint32_t i) const { return i < nwords ? w[i] : 0u; }
  __device__ __forceinline__ void refill() {
    while (nb <= 32) {
      buf |= (uint64_t)load(wi) << (32 - nb);
      wi++;
      nb += 32;
    }
  }
  __device__ __forceinline__ void init(uint32_t pos) {
    wi = pos >> 5;
    const int o = pos & 31;
    buf = (uint64_t)load(wi) << (32 + o);
    nb = 32 - o;
    wi++;
    refill();
  }
  __device__ __forceinline__ void consume(int L) {
    buf <<= L;
    nb -= L;
    if (nb <= 32) refill();
  }
};

// one symbol at the reader's position; returns its length, 0 for an invalid code
__device__ __forceinline__ int huff_sym(const HuffTables& T, const BitReader& r, uint32_t& sym) {
  const uint32_t p16 = (uint32_t)(r.buf >> 48);
  const uint32_t e = T.lut[p16 >> (16 - HP_LUT_BITS)];
  if (e) {
    sym = e & 0xffu;
    return (int)(e >> 8);
  }
  for (int L = HP_LUT_BITS + 1; L <= 16; L++) {
    const uint32_t c = p16 >> (16 - L);
    if (T.count[L] && c - T.first[L] < T.count[L]) {
      sym = T.sorted[T.index[L] + (c - T.first[L])];
      return L;
    }
  }
  return 0;
}

// number of marked bits in [a, b)
__device__ __forceinline__ uint32_t map_count(const uint32_t* map, uint32_t a, uint32_t b) {
  uint32_t n = 0;
  while (a < b) {
    const uint32_t w = a >> 5, o = a & 31, k = min(32u - o, b - a);
    const uint32_t m = (k == 32 ? 0xffffffffu : ((1u << k) - 1u)) << o;
    n += __popc(map[w] & m);
    a += k;
  }
  return n;
}

// A run of zero bits at the reader is a run of the one-bit code "0" when the
// code has one (canonical codes: the first code of length 1 is 0, symbol
// sorted[0]); the passes below take up to 32 of its codewords at once.
__device__ __forceinline__ uint32_t zero_run(const HuffTables& T, const BitReader& r,
                                             uint32_t limit) {
  if (T.count[1] == 0 || (r.buf >> 63)) return 0u;
  return min(min((uint32_t)__clzll((long long)r.buf), 32u), limit);
}

// write the n symbols decoded from bit `pos` to dst[o ..)
__device__ __forceinline__ bool huff_emit(const HuffTables& T, BitReader& rd, uint32_t pos,
                                          uint32_t n, uint8_t* __restrict__ dst, uint32_t o) {
  rd.init(pos);
  uint32_t acc = 0, p = o;
  auto put = [&](uint32_t sym) {
    acc |= sym << (8 * (p & 3));
    if ((p & 3) == 3) {
      if (p - 3 >= o) reinterpret_cast<uint32_t*>(dst)[p >> 2] = acc;
      else
        for (uint32_t q = o; q <= p; q++) dst[q] = (uint8_t)(acc >> (8 * (q & 3)));
      acc = 0;
    }
    p++;
  };
  const uint32_t z0 = T.sorted[0];
  for (uint32_t k = 0; k < n;) {
    const uint32_t run = zero_run(T, rd, n - k);
    if (run) {
      for (uint32_t q = 0; q < run; q++) put(z0);
      rd.consume((int)run);
      k += run;
      continue;
    }
    uint32_t sym;
    const int L = huff_sym(T, rd, sym);
    if (!L) return false;
    rd.consume(L);
    put(sym);
    k++;
  }
  if (p & 3)
    for (uint32_t q = max(o, p & ~3u); q < p; q++) dst[q] = (uint8_t)(acc >> (8 * (q & 3)));
  return true;
}

__device__ void huff_decode_chunk(const uint8_t* __restrict__ stored, const GroupMeta* gm,
                                  uint32_t cl, uint32_t len, uint8_t* __restrict__ dst,
                                  HuffTables& T, uint32_t* scratch, FieldMeta* meta,
                                  bool tables_ready) {
  const int tid = threadIdx.x, lane = tid & 31, NT = blockDim.x;
  const uint32_t nc = gm->nchunks;
  const uint64_t hdr = 272 + 4ull * (nc + 1);
  const bool ok = gm->stored_len >= hdr && *reinterpret_cast<const uint64_t*>(stored) == gm->S &&
                  *reinterpret_cast<const uint32_t*>(stored + 8) == HP_CHUNK &&
                  *reinterpret_cast<const uint32_t*>(stored + 12) == nc;
  if (!ok) {  // same outcome in every thread
    if (tid == 0) set_corrupt(meta);
    return;
  }
  const uint8_t* lens = stored + 16;
  const uint32_t* offs = reinterpret_cast<const uint32_t*>(stored + 272);
  const uint32_t w0 = offs[cl], w1 = offs[cl + 1];
  const uint64_t words = (gm->stored_len - hdr) / 4;
  if (w0 > w1 || w1 > words) {  // same outcome in every thread
    if (tid == 0) set_corrupt(meta);
    return;
  }
  // ---- 1. decoding tables (all threads), the gcd of the code lengths; kept
  // from the previous chunk when that one belonged to the same group
  __shared__ uint32_t s_flag, s_gl;
  if (!tables_ready) {
    // thread tid takes symbols tid + r NT (r < HP_DEC_SYMS): lengths counted per
    // warp (warp matches), ranks among equal lengths from those counts,
    // canonical first codes by one thread, then the lookup table entry by entry
    __shared__ uint32_t s_wc[HP_DEC_SYMS][HP_DEC_THREADS / 32][17];
    __shared__ uint32_t s_cnt[17];
    const int w = tid >> 5, nw = NT >> 5;
    for (int i = tid; i < HP_DEC_SYMS * (HP_DEC_THREADS / 32) * 17; i += NT) (&s_wc[0][0][0])[i] = 0;
    __syncthreads();
    uint32_t myL[HP_DEC_SYMS], rank[HP_DEC_SYMS];
    bool bad = false;
#pragma unroll
    for (int r = 0; r < HP_DEC_SYMS; r++) {
      const int sym = tid + r * HP_DEC_THREADS;
      myL[r] = sym < 256 ? lens[sym] : 0u;  // no such symbol: no code
      bad |= myL[r] > 16;
      const unsigned m = __match_any_sync(HP_FULL, myL[r]);
      rank[r] = __popc(m & ((1u << lane) - 1u));
      if ((int)(__ffs(m) - 1) == lane && myL[r] <= 16) s_wc[r][w][myL[r]] = __popc(m);
    }
    bad = __syncthreads_or(bad ? 1 : 0) != 0;
    if (tid >= 1 && tid <= 16) {  // codes of each length, one thread per length
      uint32_t n = 0;
      for (int r = 0; r < HP_DEC_SYMS; r++)
        for (int k = 0; k < nw; k++) n += s_wc[r][k][tid];
      s_cnt[tid] = n;
    }
    __syncthreads();
    if (tid == 0) {  // canonical first codes and the gcd of the lengths in use
      uint32_t c = 0, idx = 0, g = 0;
      for (int L = 1; L <= 16; L++) {
        const uint32_t n = s_cnt[L];
        T.count[L] = n;
        T.first[L] = c;
        T.index[L] = idx;
        idx += n;
        c = (c + n) << 1;
        if (n) {
          uint32_t x = g, y = (uint32_t)L;
          while (y) {
            const uint32_t tt = x % y;
            x = y;
            y = tt;
          }
          g = x;
        }
      }
      T.count[0] = 0;
      s_flag = bad ? 1u : 0u;
      s_gl = g ? g : 1u;
    }
    __syncthreads();
    if (s_flag) {
      if (tid == 0) set_corrupt(meta);
      return;
    }
#pragma unroll
    for (int r = 0; r < HP_DEC_SYMS; r++) {  // symbol order = (r, warp, lane) order
      const uint32_t L = myL[r];
      if (L) {
        uint32_t before = rank[r];
        for (int rr = 0; rr <= r; rr++)
          for (int k = 0; k < (rr < r ? nw : w); k++) before += s_wc[rr][k][L];
        T.sorted[T.index[L] + before] = (uint8_t)(tid + r * HP_DEC_THREADS);
      }
    }
    __syncthreads();
    // entry e holds the code of length L <= HP_LUT_BITS that prefixes it, if any
    for (int e = tid; e < (1 << HP_LUT_BITS); e += NT) {
      uint16_t v = 0;
      for (int L = 1; L <= HP_LUT_BITS; L++) {
        const uint32_t c = (uint32_t)e >> (HP_LUT_BITS - L);
        if (c - T.first[L] < T.count[L]) {
          v = (uint16_t)((L << 8) | T.sorted[T.index[L] + (c - T.first[L])]);
          break;
        }
      }
      T.lut[e] = v;
    }
  } else if (s_flag) {  // the group's tables were found corrupt
    if (tid == 0) set_corrupt(meta);
    return;
  }
  const uint32_t nwords = w1 - w0, nbits = nwords * 32;
  for (uint32_t i = tid; i < nwords && i < HP_MAP_WORDS; i += NT) T.map[i] = 0u;
  __syncthreads();
  BitReader rd;
  rd.w = reinterpret_cast<const uint32_t*>(stored + hdr) + w0;
  rd.nwords = nwords;
  if (nbits > HP_MAP_WORDS * 32) {  // impossible for a valid chunk: one thread, then checks
    bool fail = false;
    if (tid == 0) fail = !huff_emit(T, rd, 0, len, dst, 0);
    if (tid == 0 && fail) set_corrupt(meta);
    return;
  }
  // ---- 2. speculative decoding of NT segments on the gcd lattice, marking starts
  const uint32_t gl = s_gl, seg = (nbits + NT - 1) / NT;
  auto seg_start = [&](int i) -> uint32_t {
    return i >= NT ? nbits : min((uint32_t)i * seg, nbits) / gl * gl;
  };
  const uint32_t s_me = seg_start(tid), s_next = seg_start(tid + 1);
  uint32_t c_me = 0, e_me = s_me;
  {
    uint32_t pos = s_me;
    rd.init(pos);
    while (pos < s_next) {
      const uint32_t run = zero_run(T, rd, s_next - pos);
      if (run) {  // run starts pos .. pos + run - 1, all before s_next
        const uint64_t m = ((1ull << run) - 1ull) << (pos & 31);
        atomicOr(&T.map[pos >> 5], (uint32_t)m);
        if (m >> 32) atomicOr(&T.map[(pos >> 5) + 1], (uint32_t)(m >> 32));
        rd.consume((int)run);
        pos += run;
        c_me += run;
        continue;
      }
      uint32_t sym;
      const int L = huff_sym(T, rd, sym);
      if (!L) break;
      atomicOr(&T.map[pos >> 5], 1u << (pos & 31));
      rd.consume(L);
      pos += L;
      c_me++;
    }
    e_me = pos;
  }
  __syncthreads();
  // ---- 3. every segment's parse continues past its end until it lands on a
  // codeword start marked by a later segment's parse (from there on the two
  // agree) or runs off the data; jseg = the segment of that start (NT: none)
  uint32_t J = e_me, dj = 0, jseg = NT;
  if (tid + 1 < NT && e_me >= s_next) {
    BitReader tr = rd;
    uint32_t p = e_me, k = tid + 1;  // k: the segment holding p
    tr.init(p);
    while (p < nbits) {
      const uint32_t run = zero_run(T, tr, nbits - p);
      if (run) {  // the first marked start among the run's, if any
        const uint32_t wi = p >> 5;
        const uint64_t two = (uint64_t)T.map[wi] | (wi + 1 < nwords ? (uint64_t)T.map[wi + 1] << 32 : 0ull);
        const uint64_t hit = (two >> (p & 31)) & ((1ull << run) - 1ull);
        const uint32_t adv = hit ? (uint32_t)(__ffsll((long long)hit) - 1) : run;
        p += adv;
        dj += adv;
        if (hit) {
          while (k + 1 < (uint32_t)NT && p >= seg_start(k + 1)) k++;
          jseg = k;
          break;
        }
        tr.consume((int)run);
        continue;
      }
      while (k + 1 < (uint32_t)NT && p >= seg_start(k + 1)) k++;
      if ((T.map[p >> 5] >> (p & 31)) & 1u) {
        jseg = k;
        break;
      }
      uint32_t sym;
      const int L = huff_sym(T, tr, sym);
      if (!L) break;
      tr.consume(L);
      p += L;
      dj++;
    }
    J = p;
  }
  // The true parse is segment 0's; a segment whose parse is true hands over, at
  // its join, to the segment holding the join, whose parse is true from there
  // (induction along this chain).  Chain segments emit from their true start
  // through their join; the others emit nothing.
  __shared__ uint32_t s_J[HP_DEC_THREADS], s_seg[HP_DEC_THREADS], s_t[HP_DEC_THREADS];
  s_J[tid] = J;
  s_seg[tid] = jseg;
  s_t[tid] = 0xffffffffu;
  // (a segment reaching the data end needs no successor)
  const bool adjacent =
      __syncthreads_and(jseg == (uint32_t)tid + 1 || tid + 1 == NT || s_next >= nbits) != 0;
  uint32_t t_me;
  if (adjacent) {  // the usual case: every segment joins the next one
    t_me = tid == 0 ? 0u : s_J[tid - 1];
  } else {
    // the chain from segment 0 by pointer doubling: after round r every segment
    // within 2^(r+1) - 1 hand-overs of segment 0 is marked
    __shared__ uint32_t s_on[HP_DEC_THREADS];
    uint32_t p = jseg;
    s_on[tid] = tid == 0 ? 1u : 0u;
    __syncthreads();
    for (int r = 0; (1 << r) < NT; r++) {
      if (s_on[tid] && p < (uint32_t)NT) s_on[p] = 1u;
      const uint32_t q = p < (uint32_t)NT ? s_seg[p] : (uint32_t)NT;
      __syncthreads();
      p = q;
      s_seg[tid] = p;
      __syncthreads();
    }
    if (s_on[tid] && jseg < (uint32_t)NT) s_t[jseg] = J;  // the successor starts at the join
    if (tid == 0) s_t[0] = 0u;
    __syncthreads();
    t_me = s_t[tid];
  }
  // true symbols of this segment's emit range: its own from t_me, then the
  // continuation up to the join (none for a segment past the data end)
  const uint32_t tc_me =
      (t_me == 0xffffffffu || s_me >= nbits) ? 0u : c_me - map_count(T.map, s_me, t_me) + dj;
  // ---- 4. output offsets and the final decoding
  uint32_t total_tc;
  const uint32_t o = block_exscan(tc_me, scratch, total_tc);
  const uint32_t n_me = o < len ? min(tc_me, len - o) : 0u;
  bool fail = false;
  if (n_me) fail = !huff_emit(T, rd, t_me, n_me, dst, o);
  uint32_t total;
  (void)block_exscan(n_me, scratch, total);
  const int any_fail = __syncthreads_or(fail ? 1 : 0);
  if (any_fail || total != len) {
    if (tid == 0) set_corrupt(meta);
  }
}

// one (byte, LEB128(run-1)) record starting at s; returns its length in bytes,
// 0 when it does not fit below pe or its run field is malformed
__device__ __forceinline__ uint32_t rle_record(const uint8_t* __restrict__ pay, uint32_t s,
                                               uint32_t pe, uint32_t& v, uint32_t& run) {
  if (s + 1 >= pe) return 0;
  v = pay[s];
  uint32_t x = 0, q = s + 1;
  int shift = 0;
  while (true) {
    if (q >= pe || shift > 28) return 0;
    const uint32_t b = pay[q++];
    x |= (b & 127u) << shift;
    shift += 7;
    if (!(b & 128u)) break;
  }
  run = x + 1;
  return q - s;
}

// RLE decoding of one chunk by one warp.  The record stream is cut into 32
// byte segments; every lane parses its segment speculatively from the three
// possible record phases (our records are 2 or 3 bytes long), a pass over the
// lanes picks each lane's true phase from where the previous lane's records
// end, a prefix sum of the run lengths gives output offsets, and every lane
// expands its own runs.  Reads stay inside the chunk's bytes; any inconsistency
// marks the data corrupt.
__device__ void rle_decode_chunk(const uint8_t* __restrict__ stored, const GroupMeta* gm, uint32_t cl,
                                 uint32_t len, uint8_t* __restrict__ dst, FieldMeta* meta) {
  const int lane = threadIdx.x & 31;
  const uint32_t nc = gm->nchunks;
  const uint64_t hdr = 16 + 4ull * (nc + 1);
  bool ok = gm->stored_len >= hdr && *reinterpret_cast<const uint64_t*>(stored) == gm->S &&
            *reinterpret_cast<const uint32_t*>(stored + 8) == HP_CHUNK &&
            *reinterpret_cast<const uint32_t*>(stored + 12) == nc;
  if (!__all_sync(HP_FULL, ok)) {
    if (lane == 0) set_corrupt(meta);
    return;
  }
  const uint32_t* offs = reinterpret_cast<const uint32_t*>(stored + 16);
  const uint32_t p0 = offs[cl], p1 = offs[cl + 1];
  if (p0 > p1 || hdr + p1 > gm->stored_len) {
    if (lane == 0) set_corrupt(meta);
    return;
  }
  const uint8_t* pay = stored + hdr + p0;
  const uint32_t n = p1 - p0, seg = (n + 31) / 32;
  const uint32_t a = min(lane * seg, n), a_next = min((lane + 1) * seg, n);
  // speculative parses from phases 0, 1, 2
  uint32_t endp[3], outp[3];
  bool val[3];
#pragma unroll
  for (int ph = 0; ph < 3; ph++) {
    uint32_t s = a + ph, out = 0;
    bool good = true;
    while (s < a_next) {
      uint32_t v, run;
      const uint32_t L = rle_record(pay, s, n, v, run);
      if (!L) {
        good = false;
        break;
      }
      s += L;
      out += run;
    }
    endp[ph] = s;
    outp[ph] = out;
    val[ph] = good;
  }
  // true starts, lane by lane
  uint32_t t = 0, t_me = 0, nout = 0;
  bool bad = false;
  for (int i = 0; i < 32; i++) {
    if (lane == i) {
      t_me = t;
      uint32_t e = t;
      if (t >= a_next) {
        nout = 0;  // a record from the previous segment covers this one
      } else if (t - a < 3 && (t == a ? val[0] : t == a + 1 ? val[1] : val[2])) {
        // selects, not an index, keep the three parses in registers
        nout = t == a ? outp[0] : t == a + 1 ? outp[1] : outp[2];
        e = t == a ? endp[0] : t == a + 1 ? endp[1] : endp[2];
      } else {  // not one of the three phases (or malformed): parse again from t
        uint32_t s = t, out = 0;
        while (s < a_next) {
          uint32_t v, run;
          const uint32_t L = rle_record(pay, s, n, v, run);
          if (!L) {
            bad = true;
            break;
          }
          s += L;
          out += run;
        }
        nout = out;
        e = s;
      }
      t = e;
    }
    t = __shfl_sync(HP_FULL, t, i);
  }
  uint32_t o = nout;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t v = __shfl_up_sync(HP_FULL, o, d);
    if (lane >= d) o += v;
  }
  o -= nout;
  uint32_t total = nout;
#pragma unroll
  for (int d = 16; d; d >>= 1) total += __shfl_xor_sync(HP_FULL, total, d);
  bad = __any_sync(HP_FULL, bad) || total != len || t != n;
  if (bad) {
    if (lane == 0) set_corrupt(meta);
    return;
  }
  // expand this lane's runs into dst[o ..)
  uint32_t s = t_me, pos = o;
  while (s < a_next) {
    uint32_t v, run;
    const uint32_t L = rle_record(pay, s, n, v, run);
    s += L;
    uint32_t r = run;
    while (r && (pos & 3)) {
      dst[pos++] = (uint8_t)v;
      r--;
    }
    const uint32_t word = v * 0x01010101u;
    for (; r >= 4; r -= 4, pos += 4) *reinterpret_cast<uint32_t*>(dst + pos) = word;
    while (r) {
      dst[pos++] = (uint8_t)v;
      r--;
    }
  }
}

// one 16 KiB chunk of a newly fetched group (item = its index in the
// retrieval's list of chunks to decode)
__device__ __forceinline__ void decode_item(const uint8_t* __restrict__ slots, FieldMeta* meta,
                                            const RetrieveDev* __restrict__ rd,
                                            uint8_t* __restrict__ planes, uint32_t item,
                                            HuffTables& T, uint32_t* scratch,
                                            const GroupMeta** s_tab) {
  const uint32_t ngr = rd->n_new;
  const int ng = meta->ngroups;
  // newly fetched group holding this item: last k with new_pref[k] <= item
  uint32_t lo = 0, hi = ngr;
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) / 2;
    if (rd->new_pref[mid] <= item) lo = mid;
    else hi = mid;
  }
  const uint32_t gi = rd->new_gi[lo];
  const GroupMeta* gm = &meta->grp[gi / ng][gi % ng];
  const uint32_t cl = item - rd->new_pref[lo];
  const uint64_t start = (uint64_t)cl * HP_CHUNK, rest = gm->S - start;
  const uint32_t len = (uint32_t)(rest < HP_CHUNK ? rest : HP_CHUNK);
  const uint8_t* stored = slots + gm->slot_off;
  uint8_t* dst = planes + gm->plane_off + start;
  if (gm->method == 1) {
    const bool ready = *s_tab == gm;  // T holds this group's tables
    __syncthreads();                  // every thread has read s_tab
    huff_decode_chunk(stored, gm, cl, len, dst, T, scratch, meta, ready);
    if (threadIdx.x == 0) *s_tab = gm;
  } else if (gm->method == 2) {
    if (threadIdx.x < 32) rle_decode_chunk(stored, gm, cl, len, dst, meta);
  } else {  // direct copy of a DC group held in the slots of a compact handle
    const uint4* src = reinterpret_cast<const uint4*>(stored + start);
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (uint32_t i = threadIdx.x; i < len / 16; i += blockDim.x) d[i] = src[i];
  }
}

__global__ void __launch_bounds__(HP_DEC_THREADS) k_decode(const uint8_t* __restrict__ slots,
                                                           FieldMeta* meta,
                                                           const RetrieveDev* __restrict__ rd,
                                                           uint8_t* __restrict__ planes) {
  hp::pdl_enter();
  extern __shared__ __align__(16) unsigned char dec_smem[];
  HuffTables& T = *reinterpret_cast<HuffTables*>(dec_smem);
  __shared__ uint32_t scratch[HP_DEC_THREADS / 32];
  __shared__ const GroupMeta* s_tab;
  if (threadIdx.x == 0) s_tab = nullptr;
  __syncthreads();
  // consecutive chunks per CTA: a group's chunks mostly share its CTA's tables
  const uint32_t total = rd->items, per = (total + gridDim.x - 1) / gridDim.x;
  const uint32_t i0 = blockIdx.x * per, i1 = min(total, i0 + per);
  for (uint32_t item = i0; item < i1; item++) {
    decode_item(slots, meta, rd, planes, item, T, scratch, &s_tab);
    __syncthreads();
  }
}

void launch_decode(const uint8_t* slots, FieldMeta* meta, const RetrieveDev* rd,
                   uint32_t max_items, uint8_t* planes, cstream s) {
  if (max_items == 0) return;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = sizeof(HuffTables);
  set_smem_once((const void*)k_decode, (int)smem);
  // one wave of resident CTAs: every CTA decodes the same number of consecutive
  // chunks, so CTAs beyond the resident ones would double the launch's time
  static const int resident = [smem] {  // (thread-safe one-time initialisation)
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_decode, HP_DEC_THREADS, smem) !=
            cudaSuccess || per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
    return per_sm;
  }();
  uint32_t blocks = max_items, cap = (uint32_t)sms * (uint32_t)resident;
  if (blocks > cap) blocks = cap;
  hp::note_launch(), hp::launch_pdl(k_decode, blocks, HP_DEC_THREADS, smem, s, slots, meta, rd,
                                    planes);
}

// ------------------------------------------------------------------ batched
// unit = one chunk (or one group) of one job, one CTA each
#define HP_BATCH_UNITS(BODY)                                      \
  for (uint32_t u = blockIdx.x; u < total; u += gridDim.x) {      \
    const uint32_t j = unit_owner(unit0, njobs, u);               \
    const BatchJob& J = jobs[j];                                  \
    const uint32_t local = u - unit0[j];                          \
    BODY;                                                         \
    __syncthreads();                                              \
  }

#define HP_BATCH_PARAMS                                                                     \
  const BatchJob* __restrict__ jobs, const uint32_t* __restrict__ unit0, uint32_t njobs, \
      uint32_t total

__global__ void __launch_bounds__(256) kb_chunk_stats(HP_BATCH_PARAMS) {
  hp::pdl_enter();
  HP_BATCH_UNITS(chunk_stats_unit(J.planes, J.meta, J.chunk_group, J.hist, J.gcost, J.ccost, local))
}
__global__ void __launch_bounds__(256) kb_decide(HP_BATCH_PARAMS, uint64_t Ts, uint32_t cr_num,
                                                 uint32_t cr_den, int force) {
  hp::pdl_enter();
  HP_BATCH_UNITS(decide_unit(J.meta, J.hist, J.gcost, J.lens, Ts, cr_num, cr_den, force, local))
}
__global__ void __launch_bounds__(256) kb_huff_bits(HP_BATCH_PARAMS) {
  hp::pdl_enter();
  HP_BATCH_UNITS(huff_bits_unit(J.planes, J.meta, J.chunk_group, J.lens, J.cwords, local))
}
__global__ void __launch_bounds__(256) kb_group_offsets(HP_BATCH_PARAMS) {
  hp::pdl_enter();
  HP_BATCH_UNITS(group_offsets_unit(J.meta, J.cwords, J.ccost, J.cout, local))
}
__global__ void __launch_bounds__(256) kb_huff_encode(HP_BATCH_PARAMS) {
  hp::pdl_enter();
  HP_BATCH_UNITS(huff_encode_unit(J.planes, J.meta, J.chunk_group, J.lens, J.cout, J.slots, local))
}
__global__ void __launch_bounds__(256) kb_rle_encode(HP_BATCH_PARAMS) {
  hp::pdl_enter();
  HP_BATCH_UNITS(rle_encode_unit(J.planes, J.meta, J.chunk_group, J.cout, J.slots, local))
}
__global__ void __launch_bounds__(256) kb_headers(HP_BATCH_PARAMS) {
  hp::pdl_enter();
  HP_BATCH_UNITS(headers_unit(J.meta, J.lens, J.cout, J.slots, local))
}

static uint32_t cap_grid(uint32_t grid, uint32_t total) { return grid < total ? grid : total; }

void launch_b_chunk_stats(const BatchJob* jobs, const uint32_t* unit0, uint32_t njobs,
                          uint32_t total, uint32_t grid, cstream s) {
  if (total)
    hp::note_launch(), hp::launch_pdl(kb_chunk_stats, cap_grid(grid, total), 256, 0, s, jobs, unit0,
                                      njobs, total);
}
void launch_b_decide(const BatchJob* jobs, const uint32_t* unit0, uint32_t njobs, uint32_t total,
                     uint64_t Ts, uint32_t cr_num, uint32_t cr_den, int force, uint32_t grid,
                     cstream s) {
  if (total)
    hp::note_launch(), hp::launch_pdl(kb_decide, cap_grid(grid, total), 256, 0, s, jobs, unit0, njobs, total, Ts,
                                                                       cr_num, cr_den, force);
}
void launch_b_huff_bits(const BatchJob* jobs, const uint32_t* unit0, uint32_t njobs,
                        uint32_t total, uint32_t grid, cstream s) {
  if (total)
    hp::note_launch(), hp::launch_pdl(kb_huff_bits, cap_grid(grid, total), 256, 0, s, jobs, unit0,
                                      njobs, total);
}
void launch_b_group_offsets(const BatchJob* jobs, const uint32_t* unit0, uint32_t njobs,
                            uint32_t total, uint32_t grid, cstream s) {
  if (total)
    hp::note_launch(), hp::launch_pdl(kb_group_offsets, cap_grid(grid, total), 256, 0, s, jobs,
                                      unit0, njobs, total);
}
void launch_b_huff_encode(const BatchJob* jobs, const uint32_t* unit0, uint32_t njobs,
                          uint32_t total, uint32_t grid, cstream s) {
  if (total)
    hp::note_launch(), hp::launch_pdl(kb_huff_encode, cap_grid(grid, total), 256, 0, s, jobs, unit0,
                                      njobs, total);
}
void launch_b_rle_encode(const BatchJob* jobs, const uint32_t* unit0, uint32_t njobs,
                         uint32_t total, uint32_t grid, cstream s) {
  if (total)
    hp::note_launch(), hp::launch_pdl(kb_rle_encode, cap_grid(grid, total), 256, 0, s, jobs, unit0,
                                      njobs, total);
}
void launch_b_headers(const BatchJob* jobs, const uint32_t* unit0, uint32_t njobs, uint32_t total,
                      uint32_t grid, cstream s) {
  if (total)
    hp::note_launch(), hp::launch_pdl(kb_headers, cap_grid(grid, total), 256, 0, s, jobs, unit0,
                                      njobs, total);
}

// decode: unit = one item (chunk to decode) of one job; the per-job item
// counts are known only after the selection, so unit0 is computed on the device
__global__ void kb_items_prefix(const BatchJob* __restrict__ jobs, uint32_t njobs, uint32_t* unit0) {
  hp::pdl_enter();
  if (threadIdx.x != 0) return;
  uint32_t run = 0;
  for (uint32_t j = 0; j < njobs; j++) {
    unit0[j] = run;
    const RetrieveDev* rd = jobs[j].rd;
    if (rd->status == 0 || rd->status == -5) run += rd->items;
  }
  unit0[njobs] = run;
}

void launch_b_items_prefix(const BatchJob* jobs, uint32_t njobs, uint32_t* unit0_out, cstream s) {
  hp::note_launch(), hp::launch_pdl(kb_items_prefix, 1, 32, 0, s, jobs, njobs, unit0_out);
}

__global__ void __launch_bounds__(HP_DEC_THREADS) kb_decode(const BatchJob* __restrict__ jobs,
                                                            const uint32_t* __restrict__ unit0,
                                                            uint32_t njobs) {
  hp::pdl_enter();
  extern __shared__ __align__(16) unsigned char dec_smem[];
  HuffTables& T = *reinterpret_cast<HuffTables*>(dec_smem);
  __shared__ uint32_t scratch[HP_DEC_THREADS / 32];
  __shared__ const GroupMeta* s_tab;
  if (threadIdx.x == 0) s_tab = nullptr;
  __syncthreads();
  const uint32_t total = unit0[njobs];
  for (uint32_t u = blockIdx.x; u < total; u += gridDim.x) {
    const uint32_t j = unit_owner(unit0, njobs, u);
    const BatchJob& J = jobs[j];
    decode_item(J.slots, J.meta, J.rd, J.planes, u - unit0[j], T, scratch, &s_tab);
    __syncthreads();
  }
}

void launch_b_decode(const BatchJob* jobs, const uint32_t* unit0_dev, uint32_t njobs,
                     uint32_t grid, cstream s) {
  const size_t smem = sizeof(HuffTables);
  set_smem_once((const void*)kb_decode, (int)smem);
  hp::note_launch(), hp::launch_pdl(kb_decode, grid, HP_DEC_THREADS, smem, s, jobs, unit0_dev,
                                    njobs);
}

}  // namespace hp
