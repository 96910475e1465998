// hpmdr_encode_group_noalloc: the hybrid group encoder of hpmdr_encode_group
// (Huffman / RLE / direct copy, the same bytes and the same method choice) for
// callers that cannot allocate device memory.
//
// Who needs it: code that compresses from inside a memory regime it does not
// own, for example a simulation that reserved all of HBM for its own arena
// before starting, a solver that forbids cudaMalloc/cudaFree between time
// steps because they can synchronize the whole device, or a plug-in invoked
// from a caller-managed stream that must not change the process's memory
// footprint.  Such a caller passes its input and output buffers; every scratch
// byte this encoder needs lives in one statically sized device array declared
// below, so the call allocates nothing.
//
// Limits and rules:
//   - groups of at most HP_NOALLOC_MAX_BYTES (16 MiB, 1024 coder chunks); larger
//     groups are rejected with HPMDR_ERR_ARG;
//   - the array (about 70 KB) is a file-scope __device__ variable: every GPU
//     that loads this library holds it until the process exits;
//   - the first call on each device looks up the array's device address with
//     cudaGetSymbolAddress (with that device current); make that first call
//     before any stream capture;
//   - the call is synchronous: it waits on its stream for the status, the
//     method and the stored length before it returns;
//   - all calls share the one array and it keeps the last call's contents, so
//     calls that overlap on the GPU (other streams, other host threads) race
//     and must be serialized by the caller.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "../../include/hpmdr.h"
#include "dev_common.cuh"

using namespace hp;

#define HP_NOALLOC_MAX_BYTES (16u << 20)
#define HP_NOALLOC_MAX_CHUNKS (HP_NOALLOC_MAX_BYTES / HP_CHUNK)

struct NoAllocScratch {
  FieldMeta meta;
  uint32_t chunk_group[HP_NOALLOC_MAX_CHUNKS];
  uint32_t hist[256];               // the group's byte histogram
  unsigned long long cost;           // the group's exact RLE size
  uint32_t chunk_cost[HP_NOALLOC_MAX_CHUNKS];
  uint32_t words[HP_NOALLOC_MAX_CHUNKS];
  uint32_t off[HP_NOALLOC_MAX_CHUNKS];
  uint8_t lens[256];
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

// host side: the array's device address, looked up once per device
static std::mutex g_noalloc_mu;
static NoAllocScratch* g_noalloc_ptr[64];

static hpmdr_status noalloc_scratch(NoAllocScratch** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return HPMDR_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return HPMDR_ERR_CUDA;
    g_noalloc_ptr[dev] = (NoAllocScratch*)p;
  }
  *out = g_noalloc_ptr[dev];
  return HPMDR_OK;
}

// The shared array keeps the previous call's contents: reset the one-group
// metadata, the chunk map and the atomically accumulated histogram and RLE size
// before the coder kernels run.  (Per-chunk run costs, word counts and offsets
// are fully written before they are read.)
__global__ void k_noalloc_init(NoAllocScratch* sc, uint64_t S, uint64_t cap, uint32_t nchunks) {
  hp::pdl_enter();
  FieldMeta& m = sc->meta;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    m.status = 0;
    m.compact = 0;
    m.nlev = 1;
    m.ngroups = 1;
    GroupMeta& g = m.grp[0][0];
    g.S = S;
    g.plane_off = 0;
    g.slot_off = 0;
    g.cap = cap;
    g.stored_len = S;
    g.est_H = g.est_R = 0;
    g.nchunks = nchunks;
    g.chunk0 = 0;
    g.method = 0;
  }
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nchunks; c += gridDim.x * blockDim.x)
    sc->chunk_group[c] = 0;
  if (blockIdx.x == 0) {  // accumulated by atomics: must start at zero
    sc->hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) sc->cost = 0;
  }
}

extern "C" hpmdr_status hpmdr_encode_group_noalloc(const uint8_t* G, uint64_t S, int force,
                                                   uint64_t size_threshold, uint32_t cr_num,
                                                   uint32_t cr_den, uint8_t* out, uint64_t cap,
                                                   uint64_t* len, int* method, void* stream) {
  if (!G || !out || !len || S == 0 || force < -1 || force > 2 || ((uintptr_t)G & 15))
    return HPMDR_ERR_ARG;
  if (S > HP_NOALLOC_MAX_BYTES) return HPMDR_ERR_ARG;  // beyond the static scratch
  const uint64_t Ts = size_threshold ? size_threshold : 4096;
  if (!cr_num && !cr_den) cr_num = 2, cr_den = 1;
  if (!cr_num || !cr_den || cr_num < cr_den) return HPMDR_ERR_ARG;
  NoAllocScratch* sc = nullptr;
  hpmdr_status st = noalloc_scratch(&sc);
  if (st != HPMDR_OK) return st;
  const cudaStream_t s = (cudaStream_t)stream;
  const uint32_t nc = (uint32_t)((S + HP_CHUNK - 1) / HP_CHUNK);
  hp::note_launch(), hp::launch_pdl(k_noalloc_init, 1, 256, 0, s, sc, S, cap, nc);
  // a failed launch would leave the previous call's metadata in the array, and
  // its status, method and length would be read back as this call's
  if (cudaGetLastError() != cudaSuccess) return HPMDR_ERR_CUDA;
  ChunkMap cm{sc->chunk_group, nc};
  FieldMeta* m = &sc->meta;
  launch_chunk_stats(G, m, cm, sc->hist, &sc->cost, sc->chunk_cost, s);
  launch_decide(m, 1, sc->hist, &sc->cost, sc->lens, Ts, cr_num, cr_den, force, s);
  launch_huff_bits(G, m, cm, sc->lens, sc->words, s);
  launch_group_offsets(m, 1, sc->words, sc->chunk_cost, sc->off, s);
  launch_huff_encode(G, m, cm, sc->lens, sc->off, out, s);
  launch_rle_encode(G, m, cm, sc->off, out, s);
  launch_headers(m, 1, sc->lens, sc->off, out, s);
  if (cudaGetLastError() != cudaSuccess) return HPMDR_ERR_CUDA;
  int32_t mstatus = 0, meth = 0;
  uint64_t stored = 0;
  if (cudaMemcpyAsync(&mstatus, &m->status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&meth, &m->grp[0][0].method, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&stored, &m->grp[0][0].stored_len, 8, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return HPMDR_ERR_CUDA;
  *len = stored;
  if (method) *method = meth;
  if (mstatus) return HPMDR_ERR_ARG;  // the coded bytes did not fit in cap
  if (meth == HPMDR_DC) {
    if (cap < S) return HPMDR_ERR_ARG;
    if (cudaMemcpyAsync(out, G, S, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return HPMDR_ERR_CUDA;
  }
  return HPMDR_OK;
}
