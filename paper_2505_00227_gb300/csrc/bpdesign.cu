// The bitplane encoder designs of Sec. 4 side by side, for B = 32: the
// locality block (Sec. 4.1), register shuffling with the four warp
// instructions of Sec. 4.2 (ballot, shift tree, match-any, reduce), and the
// register block (Sec. 4.3), which is the production encoder
// (k_bitplane_encode / k_bitplane_decode).  Every design writes the same
// layout: plane 0 = sign, plane 1 + p = bit 31 - p, element j at word j >> 5,
// bit j & 31, W = 4 ceil(n / 128) words per plane, padding bits zero; decoding
// keeps the top k magnitude planes (and the sign plane when k > 0).
//
// Locality block: a thread owns the 32 contiguous elements of one word and
// moves their bits one at a time (loads strided across the warp, stores
// coalesced).  Register shuffling: a thread owns one element, a warp one word;
// each plane's word is assembled by warp communication and kept by its storing
// lane (lane p & 31; the shift tree leaves it in lane 0, which stores it).
#include "dev_common.cuh"

namespace hp {

constexpr int BPD_LOCALITY = 1, BPD_BALLOT = 2, BPD_SHIFT = 3, BPD_MATCH = 4, BPD_REDUCE = 5;

__global__ void __launch_bounds__(128) k_bpd_locality_encode(const uint32_t* __restrict__ q,
                                                             const uint8_t* __restrict__ sign,
                                                             uint32_t n, uint32_t W,
                                                             uint32_t* __restrict__ P) {
  hp::pdl_enter();
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;  // word
  if (t >= W) return;
  const uint64_t j0 = (uint64_t)t * 32;
  uint32_t v[32], s = 0;
  if (j0 + 32 <= n) {
    const uint4* q4 = reinterpret_cast<const uint4*>(q + j0);
#pragma unroll
    for (int i = 0; i < 8; i++) {
      const uint4 x = __ldg(q4 + i);
      v[4 * i] = x.x;
      v[4 * i + 1] = x.y;
      v[4 * i + 2] = x.z;
      v[4 * i + 3] = x.w;
    }
#pragma unroll
    for (int i = 0; i < 32; i++) s |= (sign[j0 + i] != 0 ? 1u : 0u) << i;
  } else {
#pragma unroll
    for (int i = 0; i < 32; i++) {
      const bool in = j0 + i < n;
      v[i] = in ? q[j0 + i] : 0u;
      s |= (in && sign[j0 + i] != 0 ? 1u : 0u) << i;
    }
  }
  P[t] = s;
#pragma unroll
  for (int p = 0; p < 32; p++) {
    uint32_t w = 0;
#pragma unroll
    for (int i = 0; i < 32; i++) w |= ((v[i] >> (31 - p)) & 1u) << i;
    P[(size_t)(1 + p) * W + t] = w;
  }
}

__global__ void __launch_bounds__(128) k_bpd_locality_decode(const uint32_t* __restrict__ P,
                                                             uint32_t n, uint32_t W, int k,
                                                             uint32_t* __restrict__ q,
                                                             uint8_t* __restrict__ sign) {
  hp::pdl_enter();
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= W) return;
  const uint64_t j0 = (uint64_t)t * 32;
  if (j0 >= n) return;
  uint32_t w[32];
#pragma unroll
  for (int p = 0; p < 32; p++) w[p] = p < k ? __ldg(P + (size_t)(1 + p) * W + t) : 0u;
  const uint32_t s = k > 0 ? __ldg(P + t) : 0u;
  uint32_t v[32];
#pragma unroll
  for (int i = 0; i < 32; i++) {
    uint32_t x = 0;
#pragma unroll
    for (int p = 0; p < 32; p++) x |= ((w[p] >> i) & 1u) << (31 - p);
    v[i] = x;
  }
  if (j0 + 32 <= n) {
    uint4* q4 = reinterpret_cast<uint4*>(q + j0);
#pragma unroll
    for (int i = 0; i < 8; i++) q4[i] = make_uint4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
#pragma unroll
    for (int i = 0; i < 32; i++) sign[j0 + i] = (uint8_t)((s >> i) & 1u);
  } else {
    for (int i = 0; j0 + i < n; i++) {
      q[j0 + i] = v[i];
      sign[j0 + i] = (uint8_t)((s >> i) & 1u);
    }
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_bpd_shuffle_encode(const uint32_t* __restrict__ q,
                                                            const uint8_t* __restrict__ sign,
                                                            uint32_t n, uint32_t W,
                                                            uint32_t* __restrict__ P) {
  hp::pdl_enter();
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t lane = threadIdx.x & 31, word = (uint32_t)(g >> 5);
  if (word >= W) return;  // whole warps: blockDim is a multiple of 32
  const bool in = g < n;
  const uint32_t x = in ? q[g] : 0u, sg = in && sign[g] != 0 ? 1u : 0u;
  uint32_t mine = 0, mine32 = 0;  // planes lane and 32 of the storing lanes
#pragma unroll
  for (int p = 0; p < 33; p++) {
    const uint32_t bit = p == 0 ? sg : (x >> (32 - p)) & 1u;
    uint32_t w;
    if (D == BPD_SHIFT) {  // tree of shifted ORs towards lane 0, which stores
      w = bit << lane;
#pragma unroll
      for (int off = 16; off; off >>= 1) w |= __shfl_down_sync(HP_FULL, w, off);
      if (lane == 0) P[(size_t)p * W + word] = w;
      continue;
    } else if (D == BPD_BALLOT) {
      w = __ballot_sync(HP_FULL, bit);
    } else if (D == BPD_MATCH) {  // lanes holding the same bit; flipped where it is 0
      const uint32_t m = __match_any_sync(HP_FULL, bit);
      w = bit ? m : ~m;
    } else {
      w = __reduce_or_sync(HP_FULL, bit << lane);
    }
    if (p < 32) {
      if (lane == (uint32_t)p) mine = w;
    } else if (lane == 0) {
      mine32 = w;
    }
  }
  if (D != BPD_SHIFT) {
    P[(size_t)lane * W + word] = mine;
    if (lane == 0) P[(size_t)32 * W + word] = mine32;
  }
}

// the decoder of the register shuffling design: lane p loads plane p's word
// and the warp broadcasts it, one plane at a time
__global__ void __launch_bounds__(256) k_bpd_shuffle_decode(const uint32_t* __restrict__ P,
                                                            uint32_t n, uint32_t W, int k,
                                                            uint32_t* __restrict__ q,
                                                            uint8_t* __restrict__ sign) {
  hp::pdl_enter();
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t lane = threadIdx.x & 31, word = (uint32_t)(g >> 5);
  if (word >= W) return;
  const uint32_t mine = (k > 0 && (int)lane <= k) ? __ldg(P + (size_t)lane * W + word) : 0u;
  const uint32_t mine32 = (k == 32 && lane == 0) ? __ldg(P + (size_t)32 * W + word) : 0u;
  uint32_t x = 0;
  for (int p = 1; p <= k; p++) {
    const uint32_t w = __shfl_sync(HP_FULL, p < 32 ? mine : mine32, p & 31);
    x |= ((w >> lane) & 1u) << (32 - p);
  }
  const uint32_t s = k > 0 ? (__shfl_sync(HP_FULL, mine, 0) >> lane) & 1u : 0u;
  if (g < n) {
    q[g] = x;
    sign[g] = (uint8_t)s;
  }
}

// design: 0 = register block (the production kernels), 1..5 above
void launch_bpd_encode(const uint32_t* q, const uint8_t* sign, uint64_t n, int design,
                       uint32_t* planes, cstream s) {
  const uint32_t W = (uint32_t)(4 * ((n + 127) / 128));
  if (design == 0) return launch_bitplane_encode(q, sign, n, 32, planes, s);
  if (design == BPD_LOCALITY) {
    hp::note_launch(), hp::launch_pdl(k_bpd_locality_encode, (W + 127) / 128, 128, 0, s, q, sign, (uint32_t)n, W,
                                                                         planes);
    return;
  }
  const uint32_t blocks = (uint32_t)(((uint64_t)W * 32 + 255) / 256);
  switch (design) {
    case BPD_BALLOT:
      hp::note_launch(), hp::launch_pdl(k_bpd_shuffle_encode<BPD_BALLOT>, blocks, 256, 0, s, q,
                                        sign, (uint32_t)n, W, planes);
      break;
    case BPD_SHIFT:
      hp::note_launch(), hp::launch_pdl(k_bpd_shuffle_encode<BPD_SHIFT>, blocks, 256, 0, s, q, sign,
                                        (uint32_t)n, W, planes);
      break;
    case BPD_MATCH:
      hp::note_launch(), hp::launch_pdl(k_bpd_shuffle_encode<BPD_MATCH>, blocks, 256, 0, s, q, sign,
                                        (uint32_t)n, W, planes);
      break;
    default:
      hp::note_launch(), hp::launch_pdl(k_bpd_shuffle_encode<BPD_REDUCE>, blocks, 256, 0, s, q,
                                        sign, (uint32_t)n, W, planes);
  }
}

void launch_bpd_decode(const uint32_t* planes, uint64_t n, int design, int k, uint32_t* q,
                       uint8_t* sign, cstream s) {
  const uint32_t W = (uint32_t)(4 * ((n + 127) / 128));
  if (design == 0) return launch_bitplane_decode(planes, n, 32, k, q, sign, s);
  if (design == BPD_LOCALITY) {
    hp::note_launch(), hp::launch_pdl(k_bpd_locality_decode, (W + 127) / 128, 128, 0, s, planes, (uint32_t)n, W, k,
                                                                         q, sign);
    return;
  }
  const uint32_t blocks = (uint32_t)(((uint64_t)W * 32 + 255) / 256);
  hp::note_launch(), hp::launch_pdl(k_bpd_shuffle_decode, blocks, 256, 0, s, planes, (uint32_t)n, W,
                                    k, q, sign);
}

}  // namespace hp
