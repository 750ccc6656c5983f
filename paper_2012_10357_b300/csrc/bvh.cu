// Device LBVH builder: instance world boxes, Morton codes, radix sort, binary
// radix tree (Karras 2012, "Maximizing parallelism in the construction of
// BVHs, octrees and k-d trees") and bottom-up box unions.
//
// The acceleration structure DXR builds for procedural geometry encloses the
// AABBs of each geometry set in a BLAS and instances BLASes in a TLAS
// (Section 2.2.3, Fig. 3; one BLAS per geometry set, Section 3.1.5). Here both
// levels are BVH2 trees whose nodes store both child boxes (64 B per node).
//
// Every floating-point step that decides an integer (centroid, quantisation)
// uses explicitly rounded single-precision operations, so codes, tree and
// boxes are bit-reproducible by a plain CPU implementation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"

namespace pr {
namespace {

__device__ __forceinline__ uint32_t part1by2(uint32_t x) {
  x &= 0x3FFu;
  x = (x | (x << 16)) & 0x030000FFu;
  x = (x | (x << 8)) & 0x0300F00Fu;
  x = (x | (x << 4)) & 0x030C30C3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

__device__ __forceinline__ const float* leaf_box(const LevelDesc& J, uint32_t k) {
  return J.boxes + 6 * (size_t)(J.gather ? J.gather[k] : k);
}

__device__ __forceinline__ float centroid(const float* b, int a) { return __fmul_rn(__fadd_rn(b[a], b[3 + a]), 0.5f); }

__device__ __forceinline__ uint32_t quantise(float c, float lo, float ext) {
  float u = ext > 0.f ? __fdiv_rn(__fsub_rn(c, lo), ext) : 0.f;
  uint32_t q = __float2uint_rz(__fmul_rn(u, 1024.f));
  return q > 1023u ? 1023u : q;
}

__device__ __forceinline__ uint32_t morton(const float* b, const float* clo, const float* ext) {
  uint32_t qx = quantise(centroid(b, 0), clo[0], ext[0]);
  uint32_t qy = quantise(centroid(b, 1), clo[1], ext[1]);
  uint32_t qz = quantise(centroid(b, 2), clo[2], ext[2]);
  return (part1by2(qx) << 2) | (part1by2(qy) << 1) | part1by2(qz);
}

// Block-wide min/max of 3 floats each (blockDim multiple of 32, <= 1024).
__device__ void block_minmax3(float lo[3], float hi[3], float* sh /* 6*32 */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = fminf(lo[a], __shfl_xor_sync(0xFFFFFFFFu, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xFFFFFFFFu, hi[a], o));
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) { sh[a * 32 + warp] = lo[a]; sh[(3 + a) * 32 + warp] = hi[a]; }
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float l = INFINITY, h = -INFINITY;
    for (int w = 0; w < nw; ++w) { l = fminf(l, sh[a * 32 + w]); h = fmaxf(h, sh[(3 + a) * 32 + w]); }
    lo[a] = l;
    hi[a] = h;
  }
  __syncthreads();
}

__device__ __forceinline__ void store_child_box(float4* node, int side, const float b[6]) {
  float* f = reinterpret_cast<float*>(node);
  int o = side * 6;
  for (int k = 0; k < 6; ++k) f[o + k] = b[k];
}

__device__ __forceinline__ void write_root(float* rb, const float b[6]) {
  rb[0] = b[0]; rb[1] = b[1]; rb[2] = b[2]; rb[3] = 0.f;
  rb[4] = b[3]; rb[5] = b[4]; rb[6] = b[5]; rb[7] = 0.f;
}

// Karras radix-tree node i over n distinct sorted keys: its key range
// [first, last] and the split gamma (left child [first, gamma]).
template <typename KeyFn>
__device__ __forceinline__ void karras_node(int i, int n, KeyFn key, int& first, int& last, int& gamma) {
  auto delta = [&](int a, int b) -> int {
    if (b < 0 || b >= n) return -1;
    return __clzll((long long)(key(a) ^ key(b)));
  };
  int d = (delta(i, i + 1) - delta(i, i - 1)) > 0 ? 1 : -1;
  int dmin = delta(i, i - d);
  int lmax = 2;
  while (delta(i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (delta(i, i + (l + t) * d) > dmin) l += t;
  int j = i + l * d;
  int dnode = delta(i, j);
  int s = 0;
  int div = 2;
  for (;;) {
    int t = (l + div - 1) / div;
    if (delta(i, i + (s + t) * d) > dnode) s += t;
    if (t <= 1) break;
    div <<= 1;
  }
  gamma = i + s * d + (d < 0 ? -1 : 0);
  first = min(i, j);
  last = max(i, j);
}

// A level of one leaf: its centroid bounds are that centroid (extent 0), so
// the leaf's Morton code is 0; the root box is the leaf's box.
__device__ void single_leaf_level(const LevelDesc& J) {
  J.perm[0] = 0u;
  J.codes[0] = 0u;
  const float* b = leaf_box(J, 0);
  const float bb[6] = {b[0], b[1], b[2], b[3], b[4], b[5]};
  write_root(J.root_box, bb);
}

// ---- single-CTA build of a small level (n <= kSmallMax) --------------------
__device__ void build_small_body(const LevelDesc& J) {
  const uint32_t n = J.n;
  if (n == 0) return;
  if (n == 1) {
    if (threadIdx.x == 0) single_leaf_level(J);
    return;
  }
  __shared__ unsigned long long keys[kSmallMax];
  __shared__ float red[6 * 32];
  __shared__ float sh_lo[3], sh_ext[3];
  const int tid = threadIdx.x, bd = blockDim.x;

  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (uint32_t k = tid; k < n; k += bd) {
    const float* b = leaf_box(J, k);
    for (int a = 0; a < 3; ++a) {
      float c = centroid(b, a);
      lo[a] = fminf(lo[a], c);
      hi[a] = fmaxf(hi[a], c);
    }
  }
  block_minmax3(lo, hi, red);
  if (tid == 0)
    for (int a = 0; a < 3; ++a) { sh_lo[a] = lo[a]; sh_ext[a] = __fsub_rn(hi[a], lo[a]); }
  __syncthreads();

  uint32_t P = 1;
  while (P < n) P <<= 1;
  for (uint32_t k = tid; k < P; k += bd) {
    if (k < n) {
      uint32_t code = morton(leaf_box(J, k), sh_lo, sh_ext);
      keys[k] = ((unsigned long long)code << 32) | k;
    } else {
      keys[k] = ~0ull;
    }
  }
  __syncthreads();
  // bitonic sort of P keys (distinct, so the order is unique)
  for (uint32_t size = 2; size <= P; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t t = tid; t < P / 2; t += bd) {
        uint32_t a = 2 * t - (t & (stride - 1));
        uint32_t b = a + stride;
        bool up = (a & size) == 0;
        unsigned long long ka = keys[a], kb = keys[b];
        if ((ka > kb) == up) { keys[a] = kb; keys[b] = ka; }
      }
      __syncthreads();
    }
  }
  for (uint32_t p = tid; p < n; p += bd) {
    J.perm[p] = (uint32_t)(keys[p] & 0xFFFFFFFFull);
    J.codes[p] = (uint32_t)(keys[p] >> 32);
  }
  auto key = [&](int a) -> unsigned long long { return keys[a]; };
  for (int i = tid; i < (int)n - 1; i += bd) {
    int first, last, g;
    karras_node(i, (int)n, key, first, last, g);
    float box[2][6];
    int ref[2];
    int rng[2][2] = {{first, g}, {g + 1, last}};
    for (int side = 0; side < 2; ++side) {
      int f = rng[side][0], l = rng[side][1];
      ref[side] = (f == l) ? (int)(kLeafBit | (J.leaf_ref_base + (uint32_t)(keys[f] & 0xFFFFFFFFull))) : (side ? f : l);
      float bl[3] = {INFINITY, INFINITY, INFINITY}, bh[3] = {-INFINITY, -INFINITY, -INFINITY};
      for (int p = f; p <= l; ++p) {
        const float* b = leaf_box(J, (uint32_t)(keys[p] & 0xFFFFFFFFull));
        for (int a = 0; a < 3; ++a) { bl[a] = fminf(bl[a], b[a]); bh[a] = fmaxf(bh[a], b[3 + a]); }
      }
      for (int a = 0; a < 3; ++a) { box[side][a] = bl[a]; box[side][3 + a] = bh[a]; }
    }
    float4* node = J.nodes + 4 * (size_t)i;
    store_child_box(node, 0, box[0]);
    store_child_box(node, 1, box[1]);
    node[3] = make_float4(__int_as_float(ref[0]), __int_as_float(ref[1]), 0.f, 0.f);
    if (i == 0) {
      float rb[6];
      for (int a = 0; a < 3; ++a) { rb[a] = fminf(box[0][a], box[1][a]); rb[3 + a] = fmaxf(box[0][3 + a], box[1][3 + a]); }
      write_root(J.root_box, rb);
    }
  }
}

__global__ void __launch_bounds__(256) k_build_small(const LevelDesc* jobs) { build_small_body(jobs[blockIdx.x]); }

__global__ void __launch_bounds__(256) k_build_small_one(LevelDesc J) { build_small_body(J); }

// ---- multi-kernel build of a large level ----------------------------------
__global__ void __launch_bounds__(256) k_centroid_partial(LevelDesc J, float* partial) {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < J.n; k += gridDim.x * blockDim.x) {
    const float* b = leaf_box(J, k);
    for (int a = 0; a < 3; ++a) {
      float c = centroid(b, a);
      lo[a] = fminf(lo[a], c);
      hi[a] = fmaxf(hi[a], c);
    }
  }
  __shared__ float red[6 * 32];
  block_minmax3(lo, hi, red);
  if (threadIdx.x == 0)
    for (int a = 0; a < 3; ++a) { partial[6 * blockIdx.x + a] = lo[a]; partial[6 * blockIdx.x + 3 + a] = hi[a]; }
}

__global__ void __launch_bounds__(256) k_morton(LevelDesc J, const float* partial, int n_partial, uint32_t* keys,
                                                 uint32_t* vals) {
  __shared__ float red[6 * 32];
  __shared__ float sh_lo[3], sh_ext[3];
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int p = threadIdx.x; p < n_partial; p += blockDim.x)
    for (int a = 0; a < 3; ++a) {
      lo[a] = fminf(lo[a], partial[6 * p + a]);
      hi[a] = fmaxf(hi[a], partial[6 * p + 3 + a]);
    }
  block_minmax3(lo, hi, red);
  if (threadIdx.x == 0)
    for (int a = 0; a < 3; ++a) { sh_lo[a] = lo[a]; sh_ext[a] = __fsub_rn(hi[a], lo[a]); }
  __syncthreads();
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < J.n; k += gridDim.x * blockDim.x) {
    keys[k] = morton(leaf_box(J, k), sh_lo, sh_ext);
    vals[k] = k;
  }
}

// Radix sort, 8-bit digits, tiles of kSortTile keys (256 threads x 8 rounds).
__global__ void __launch_bounds__(256) k_radix_hist(const uint32_t* keys, uint32_t n, int shift, uint32_t* hist,
                                                     uint32_t n_tiles) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  uint32_t base = blockIdx.x * kSortTile;
  for (uint32_t r = 0; r < kSortTile / 256; ++r) {
    uint32_t k = base + r * 256 + threadIdx.x;
    if (k < n) atomicAdd(&cnt[(keys[k] >> shift) & 0xFFu], 1u);
  }
  __syncthreads();
  hist[threadIdx.x * n_tiles + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive scan of m = 256 * n_tiles counts in digit-major order (one block).
__global__ void __launch_bounds__(1024) k_radix_scan(uint32_t* hist, uint32_t m) {
  __shared__ uint32_t sums[1024];
  const uint32_t per = (m + blockDim.x - 1) / blockDim.x;
  const uint32_t b = threadIdx.x * per, e = min(m, b + per);
  uint32_t s = 0;
  for (uint32_t i = b; i < e; ++i) s += hist[i];
  sums[threadIdx.x] = s;
  __syncthreads();
  for (uint32_t o = 1; o < blockDim.x; o <<= 1) {
    uint32_t v = threadIdx.x >= o ? sums[threadIdx.x - o] : 0u;
    __syncthreads();
    sums[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = threadIdx.x ? sums[threadIdx.x - 1] : 0u;
  for (uint32_t i = b; i < e; ++i) {
    uint32_t v = hist[i];
    hist[i] = run;
    run += v;
  }
}

// Stable scatter: within a tile, rounds in order, warps in order, lanes in
// order; equal digits keep their input order (ranks from __match_any_sync).
__global__ void __launch_bounds__(256) k_radix_scatter(const uint32_t* keys_in, const uint32_t* vals_in,
                                                        uint32_t* keys_out, uint32_t* vals_out, uint32_t n, int shift,
                                                        const uint32_t* hist, uint32_t n_tiles) {
  __shared__ uint32_t run[256];
  __shared__ uint32_t wcnt[8][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  run[tid] = hist[tid * n_tiles + blockIdx.x];
  const uint32_t base = blockIdx.x * kSortTile;
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (uint32_t r = 0; r < kSortTile / 256; ++r) {
    for (int w = 0; w < 8; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    uint32_t k = base + r * 256 + tid;
    bool valid = k < n;
    uint32_t key = valid ? keys_in[k] : 0u;
    uint32_t digit = valid ? ((key >> shift) & 0xFFu) : 256u;   // 256: invalid, never matches a digit
    uint32_t peers = __match_any_sync(0xFFFFFFFFu, digit);
    uint32_t rank = __popc(peers & lt_mask);
    if (valid && rank == 0) wcnt[warp][digit] = __popc(peers);
    __syncthreads();
    if (valid) {
      uint32_t off = run[digit] + rank;
      for (int w = 0; w < warp; ++w) off += wcnt[w][digit];
      keys_out[off] = key;
      vals_out[off] = vals_in[k];
    }
    __syncthreads();
    uint32_t tot = 0;
    for (int w = 0; w < 8; ++w) tot += wcnt[w][tid];
    run[tid] += tot;
    __syncthreads();
  }
}

// done: when set and nonzero, a PLOC launch already built the level (its fallback
// path; null for the LBVH build)
__global__ void __launch_bounds__(256) k_karras(LevelDesc J, const uint32_t* codes, const uint32_t* vals,
                                                 uint32_t* parent_int, uint32_t* parent_leaf, const uint32_t* done) {
  if (done && *done) return;
  const int n = (int)J.n;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    J.perm[i] = vals[i];
    J.codes[i] = codes[i];
  }
  if (i >= n - 1) return;
  auto key = [&](int a) -> unsigned long long { return ((unsigned long long)codes[a] << 32) | vals[a]; };
  int first, last, g;
  karras_node(i, n, key, first, last, g);
  int lref, rref;
  if (first == g) {
    lref = (int)(kLeafBit | (J.leaf_ref_base + vals[g]));
    parent_leaf[g] = (uint32_t)i;
  } else {
    lref = g;
    parent_int[g] = (uint32_t)i;
  }
  if (last == g + 1) {
    rref = (int)(kLeafBit | (J.leaf_ref_base + vals[g + 1]));
    parent_leaf[g + 1] = (uint32_t)i;
  } else {
    rref = g + 1;
    parent_int[g + 1] = (uint32_t)i;
  }
  J.nodes[4 * (size_t)i + 3] = make_float4(__int_as_float(lref), __int_as_float(rref), 0.f, 0.f);
}

// Bottom-up unions: each leaf walks up; the second arrival at a node unites
// both child boxes (Karras 2012, Section 4) and continues to the parent.
__global__ void __launch_bounds__(256) k_refit(LevelDesc J, const uint32_t* vals, const uint32_t* parent_int,
                                                const uint32_t* parent_leaf, uint32_t* counters, const uint32_t* done) {
  if (done && *done) return;
  const uint32_t n = J.n;
  uint32_t pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= n) return;
  const float* b = leaf_box(J, vals[pos]);
  float box[6] = {b[0], b[1], b[2], b[3], b[4], b[5]};
  int ref = (int)(kLeafBit | (J.leaf_ref_base + vals[pos]));
  uint32_t p = parent_leaf[pos];
  for (;;) {
    float4* node = J.nodes + 4 * (size_t)p;
    int lref = __float_as_int(__ldcg(&node[3].x));
    int side = (lref == ref) ? 0 : 1;
    store_child_box(node, side, box);
    __threadfence();
    uint32_t old = atomicAdd(&counters[p], 1u);
    if (old == 0) return;
    __threadfence();
    const float* f = reinterpret_cast<const float*>(node) + (1 - side) * 6;
    for (int a = 0; a < 3; ++a) {
      box[a] = fminf(box[a], __ldcg(f + a));
      box[3 + a] = fmaxf(box[3 + a], __ldcg(f + 3 + a));
    }
    if (p == 0) {
      write_root(J.root_box, box);
      return;
    }
    ref = (int)p;
    p = parent_int[p];
  }
}

// ---- PLOC: bottom-up clustering of a large level ---------------------------
// Parallel locally-ordered clustering (Meister & Bittner 2018): the leaves in
// Morton order are the first clusters; every round each cluster finds its
// nearest neighbour among the kPlocRadius clusters on either side: the least
// pair by the surface area of the box enclosing both, then by distance in the
// list, then with the lower index even before odd, then by the lower index.
// That is a total order on pairs, so the least pair of a round is mutual and
// every round merges at least one pair; on equal boxes it pairs 0-1, 2-3, ...
// and halves the list. Mutual nearest neighbours merge into a new node; a
// prefix sum over the survivors keeps the order. New nodes are numbered downward from n - 2, so the final
// merge is node 0, the root the traversal starts from. The node layout is
// the LBVH's, so the 4-wide collapse and the traversal take the tree as is.
constexpr int kPlocRadius = 16;
constexpr int kPlocThreads = 256;
// Rounds with at most this many clusters run in block 0 alone, with the list
// in shared memory (two lists of 32-byte records and the neighbours).
constexpr uint32_t kPlocTail = 2048;
constexpr size_t kPlocSmem = 2 * kPlocTail * 32 + kPlocTail * 4;
// A cluster is a 32-byte record: (lo.xyz, reference bits), (hi.xyz, 0).
// header words (in the radix histogram's buffer, free once the sort is done)
constexpr int kHdrOk = 0, kHdrAbort = 1, kHdrCount = 2, kHdrGen = 3;
constexpr size_t kPlocPartOffset = 256;              // bytes: per-block counts follow the header
constexpr unsigned long long kPlocWaitNs = 2000000000ull;
constexpr uint32_t kPlocMaxSpins = 1u << 25;

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of the cooperative launch (which makes every block
// resident), with a limit: a block that waits longer than kPlocWaitNs, or
// sees that another block gave up, gives up too and the kernel ends; the
// LBVH passes launched after it then build the level instead.
__device__ bool grid_barrier(uint32_t* hdr, uint32_t* error_word, uint32_t& gen, uint32_t* ok_sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t ok = 1;
    __threadfence();
    const uint32_t arrived = atomicAdd(&hdr[kHdrCount], 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&hdr[kHdrCount], 0u);
      __threadfence();
      atomicExch(&hdr[kHdrGen], gen + 1);
    } else {
      const unsigned long long t0 = global_ns();
      for (uint32_t spins = 0;; ++spins) {
        if (ld_acquire_u32(&hdr[kHdrGen]) != gen) break;
        if (ld_acquire_u32(&hdr[kHdrAbort]) || spins > kPlocMaxSpins || global_ns() - t0 > kPlocWaitNs) {
          atomicExch(&hdr[kHdrAbort], 1u);
          if (error_word) atomicOr(error_word, 1u << PR_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    *ok_sh = ok;
  }
  ++gen;
  __syncthreads();
  return *ok_sh != 0;
}

// exclusive block scan of two counters packed in a 64-bit value
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v, unsigned long long* sh,
                                                              unsigned long long& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = lane < kPlocThreads / 32 ? sh[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kPlocThreads / 32) sh[lane] = w;
  }
  __syncthreads();
  total = sh[kPlocThreads / 32 - 1];
  const unsigned long long before = warp ? sh[warp - 1] : 0ull;
  __syncthreads();
  return before + x - v;
}

__device__ __forceinline__ float rec_half_area(const float4& al, const float4& ah, const float4& bl,
                                                const float4& bh) {
  const float dx = fmaxf(ah.x, bh.x) - fminf(al.x, bl.x);
  const float dy = fmaxf(ah.y, bh.y) - fminf(al.y, bl.y);
  const float dz = fmaxf(ah.z, bh.z) - fminf(al.z, bl.z);
  const float s = fmaf(dx, dy, fmaf(dy, dz, dz * dx));
  return s == s ? s : INFINITY;   // NaN (a non-finite box) orders last
}

// Nearest neighbour of cluster i among the clusters within kPlocRadius of it
// (list of m); rec(j, lo, hi) reads cluster j's record.
template <class Rec>
__device__ __forceinline__ int ploc_nearest(uint32_t i, uint32_t m, Rec rec) {
  float4 il, ih;
  rec(i, il, ih);
  const uint32_t lo = i > (uint32_t)kPlocRadius ? i - kPlocRadius : 0u;
  const uint32_t hi = min(m - 1, i + (uint32_t)kPlocRadius);
  float best = INFINITY;
  int bj = -1;
  for (uint32_t j = lo; j <= hi; ++j) {
    if (j == i) continue;
    float4 jl, jh;
    rec(j, jl, jh);
    const float a = rec_half_area(il, ih, jl, jh);
    bool take = bj < 0 || a < best;
    if (!take && a == best) {
      const uint32_t d = j > i ? j - i : i - j, db = (uint32_t)bj > i ? (uint32_t)bj - i : i - (uint32_t)bj;
      const uint32_t l = min(i, j), lb = min(i, (uint32_t)bj);
      take = d != db ? d < db : ((l ^ lb) & 1u) ? (l & 1u) == 0u : l < lb;
    }
    if (take) {
      best = a;
      bj = (int)j;
    }
  }
  return bj;
}

// The merged node of clusters i < j (left i, right j) and the record of the new cluster.
__device__ __forceinline__ void ploc_merge(float4* nodes, uint32_t node, const float4& il, const float4& ih,
                                           const float4& jl, const float4& jh, float4& ol, float4& oh) {
  float4* nd = nodes + 4 * (size_t)node;   // the BVH2 node layout: both child boxes, then the refs
  nd[0] = make_float4(il.x, il.y, il.z, ih.x);
  nd[1] = make_float4(ih.y, ih.z, jl.x, jl.y);
  nd[2] = make_float4(jl.z, jh.x, jh.y, jh.z);
  nd[3] = make_float4(il.w, jl.w, 0.f, 0.f);
  ol = make_float4(fminf(il.x, jl.x), fminf(il.y, jl.y), fminf(il.z, jl.z), __int_as_float((int)node));
  oh = make_float4(fmaxf(ih.x, jh.x), fmaxf(ih.y, jh.y), fmaxf(ih.z, jh.z), 0.f);
}

// Flags of cluster i with neighbour j, back = nn[j]: keep (i survives the round,
// alone or as the merged node of its mutual pair), merge (i is the lower index
// of a mutual pair); packed as keep + (merge << 32).
__device__ __forceinline__ unsigned long long keep_merge(uint32_t i, int j, int back) {
  const bool mutual = back == (int)i;
  const bool keep = !(mutual && (uint32_t)j < i);
  const bool merge = mutual && i < (uint32_t)j;
  return (keep ? 1ull : 0ull) + (merge ? (1ull << 32) : 0ull);
}

// Neighbours and flags of clusters base .. base + 3 (those below end), all
// loads issued before any is used.
struct Flags4 {
  int j[4];
  unsigned long long f[4];
};
__device__ __forceinline__ Flags4 flags4(const int* nn, uint32_t base, uint32_t end) {
  Flags4 q;
  int back[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) q.j[k] = base + k < end ? __ldcg(nn + base + k) : -1;
#pragma unroll
  for (int k = 0; k < 4; ++k) back[k] = q.j[k] >= 0 ? __ldcg(nn + q.j[k]) : -1;
#pragma unroll
  for (int k = 0; k < 4; ++k) q.f[k] = base + k < end ? keep_merge(base + k, q.j[k], back[k]) : 0ull;
  return q;
}

__global__ void __launch_bounds__(kPlocThreads) k_ploc(PlocArgs A) {
  extern __shared__ float4 smem[];   // kPlocSmem bytes
  __shared__ unsigned long long sh[kPlocThreads / 32];
  __shared__ uint32_t ok_sh;
  uint32_t* hdr = A.hdr;
  const uint32_t n = A.J.n;
  uint32_t gen = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t leaf = A.vals[i];
    A.J.perm[i] = leaf;
    A.J.codes[i] = A.codes[i];
    const float* b = leaf_box(A.J, leaf);
    A.R[0][2 * (size_t)i] = make_float4(b[0], b[1], b[2], __int_as_float((int)(kLeafBit | (A.J.leaf_ref_base + leaf))));
    A.R[0][2 * (size_t)i + 1] = make_float4(b[3], b[4], b[5], 0.f);
  }
  if (!grid_barrier(hdr, A.error_word, gen, &ok_sh)) return;
  uint32_t m = n, next = n - 2;
  int cur = 0;
  const uint32_t nb = gridDim.x, bid = blockIdx.x;
  // ---- rounds over the whole grid, list in global memory
  while (m > kPlocTail) {
    const float4* R = cur ? A.R[1] : A.R[0];
    // 1. nearest neighbours, tiles of kPlocThreads clusters staged with their halo in shared memory
    const uint32_t ntiles = (m + kPlocThreads - 1) / kPlocThreads;
    constexpr int kStage = 2 * (kPlocThreads + 2 * kPlocRadius);   // float4 of a tile and its halo
    constexpr int kStagePer = (kStage + kPlocThreads - 1) / kPlocThreads;
    for (uint32_t t = bid; t < ntiles; t += nb) {
      const long long g0 = 2ll * ((long long)t * kPlocThreads - kPlocRadius);
      float4 v[kStagePer];
#pragma unroll
      for (int q = 0; q < kStagePer; ++q) {   // all loads first, then the stores
        const int k = threadIdx.x + q * kPlocThreads;
        const long long g = g0 + k;
        v[q] = (k < kStage && g >= 0 && g < 2ll * m) ? __ldcg(R + g) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < kStagePer; ++q) {
        const int k = threadIdx.x + q * kPlocThreads;
        if (k < kStage) smem[k] = v[q];
      }
      __syncthreads();
      const uint32_t i = t * kPlocThreads + threadIdx.x;
      if (i < m) {
        const uint32_t row0 = t * kPlocThreads - kPlocRadius;   // cluster of staged record 0 (wraps below 0)
        A.nn[i] = ploc_nearest(i, m, [&](uint32_t j, float4& lo, float4& hi) {
          lo = smem[2 * (j - row0)];
          hi = smem[2 * (j - row0) + 1];
        });
      }
      __syncthreads();
    }
    if (!grid_barrier(hdr, A.error_word, gen, &ok_sh)) return;
    // 2. survivors and merges of each block's chunk; a thread takes 4 consecutive clusters
    const uint32_t chunk = ((m + nb - 1) / nb + 3u) & ~3u;
    const uint32_t c0 = min(m, bid * chunk), c1 = min(m, c0 + chunk);
    unsigned long long cnt = 0;
    for (uint32_t g0 = c0; g0 < c1; g0 += 4 * kPlocThreads) {
      const Flags4 q = flags4(A.nn, g0 + 4 * threadIdx.x, c1);
      cnt += q.f[0] + q.f[1] + q.f[2] + q.f[3];
    }
    unsigned long long tot;
    block_excl_scan(cnt, sh, tot);
    if (threadIdx.x == 0) A.part[bid] = tot;
    if (!grid_barrier(hdr, A.error_word, gen, &ok_sh)) return;
    // 3. this block's exclusive prefix of the block counts and the round's totals
    unsigned long long pre_part = 0, all_part = 0;
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) {
      const unsigned long long v = __ldcg(A.part + b);
      all_part += v;
      if (b < bid) pre_part += v;
    }
    unsigned long long pre, all;
    block_excl_scan(pre_part, sh, pre);
    block_excl_scan(all_part, sh, all);
    // 4. merged nodes and the compacted list, in order
    float4* Rn = cur ? A.R[0] : A.R[1];
    unsigned long long run = pre;
    for (uint32_t g0 = c0; g0 < c1; g0 += 4 * kPlocThreads) {
      const uint32_t base = g0 + 4 * threadIdx.x;
      const Flags4 q = flags4(A.nn, base, c1);
      unsigned long long t;
      unsigned long long e = run + block_excl_scan(q.f[0] + q.f[1] + q.f[2] + q.f[3], sh, t);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (q.f[k] & 0xFFFFFFFFull) {
          const uint32_t i = base + k, pos = (uint32_t)(e & 0xFFFFFFFFull);
          float4 il = __ldcg(R + 2 * (size_t)i), ih = __ldcg(R + 2 * (size_t)i + 1);
          if (q.f[k] >> 32) {
            const float4 jl = __ldcg(R + 2 * (size_t)q.j[k]), jh = __ldcg(R + 2 * (size_t)q.j[k] + 1);
            ploc_merge(A.J.nodes, next - (uint32_t)(e >> 32), il, ih, jl, jh, il, ih);
          }
          Rn[2 * (size_t)pos] = il;
          Rn[2 * (size_t)pos + 1] = ih;
        }
        e += q.f[k];
      }
      run += t;
    }
    m = (uint32_t)(all & 0xFFFFFFFFull);
    next -= (uint32_t)(all >> 32);
    cur ^= 1;
    // (the next round writes the block counts only after its first barrier,
    // when every block has read this round's)
    if (!grid_barrier(hdr, A.error_word, gen, &ok_sh)) return;
  }
  // ---- the last rounds in block 0, list in shared memory
  if (bid != 0) return;
  float4* Lc = smem;                     // this round's list
  float4* Ln = smem + 2 * kPlocTail;     // the next round's
  int* snn = reinterpret_cast<int*>(smem + 4 * kPlocTail);
  {
    const float4* src = cur ? A.R[1] : A.R[0];
    for (uint32_t k = threadIdx.x; k < 2 * m; k += blockDim.x) Lc[k] = __ldcg(src + k);
  }
  __syncthreads();
  while (m > 1) {
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x)
      snn[i] = ploc_nearest(i, m, [&](uint32_t j, float4& lo, float4& hi) {
        lo = Lc[2 * j];
        hi = Lc[2 * j + 1];
      });
    __syncthreads();
    unsigned long long run = 0;
    for (uint32_t g0 = 0; g0 < m; g0 += 4 * kPlocThreads) {
      const uint32_t base = g0 + 4 * threadIdx.x;
      unsigned long long f[4];
      int jj[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        jj[k] = base + k < m ? snn[base + k] : -1;
        f[k] = base + k < m ? keep_merge(base + k, jj[k], snn[jj[k]]) : 0ull;
      }
      unsigned long long t;
      unsigned long long e = run + block_excl_scan(f[0] + f[1] + f[2] + f[3], sh, t);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (f[k] & 0xFFFFFFFFull) {
          const uint32_t i = base + k, pos = (uint32_t)(e & 0xFFFFFFFFull);
          float4 il = Lc[2 * i], ih = Lc[2 * i + 1];
          if (f[k] >> 32)
            ploc_merge(A.J.nodes, next - (uint32_t)(e >> 32), il, ih, Lc[2 * jj[k]], Lc[2 * jj[k] + 1], il, ih);
          Ln[2 * pos] = il;
          Ln[2 * pos + 1] = ih;
        }
        e += f[k];
      }
      run += t;
    }
    __syncthreads();
    m = (uint32_t)(run & 0xFFFFFFFFull);
    next -= (uint32_t)(run >> 32);
    float4* tmp = Lc;
    Lc = Ln;
    Ln = tmp;
  }
  if (threadIdx.x == 0) {
    const float4 lo = Lc[0], hi = Lc[1];
    const float box[6] = {lo.x, lo.y, lo.z, hi.x, hi.y, hi.z};
    write_root(A.J.root_box, box);
    hdr[kHdrOk] = 1u;
  }
}

// Instance k: world box of its BLAS root box, world->object transform, record.
__device__ void instance_body(uint32_t k, const InstanceArgs& A) {
  const float* xform = A.xform;
  const uint32_t *inst_blas = A.inst_blas, *inst_id = A.inst_id, *inst_sbt = A.inst_sbt, *inst_mask = A.inst_mask;
  const float4* blas_box = A.blas_box;
  const int4* blas_info = A.blas_info;
  float* boxes = A.boxes;
  float4* rec = A.rec;
  const float* m = xform + 12 * (size_t)k;
  uint32_t b = inst_blas[k];
  float4 blo = blas_box[2 * b], bhi = blas_box[2 * b + 1];
  float rl[3] = {blo.x, blo.y, blo.z}, rh[3] = {bhi.x, bhi.y, bhi.z};
  // world box: per axis t_i + sum_j min/max(m_ij lo_j, m_ij hi_j), j = 0,1,2 in order
  for (int i = 0; i < 3; ++i) {
    float lo = m[4 * i + 3], hi = m[4 * i + 3];
    for (int j = 0; j < 3; ++j) {
      float a = __fmul_rn(m[4 * i + j], rl[j]);
      float c = __fmul_rn(m[4 * i + j], rh[j]);
      lo = __fadd_rn(lo, fminf(a, c));
      hi = __fadd_rn(hi, fmaxf(a, c));
    }
    boxes[6 * (size_t)k + i] = lo;
    boxes[6 * (size_t)k + 3 + i] = hi;
  }
  // world -> object: inverse of the 3x3 part by its adjugate, t' = -L^-1 t
  float a00 = m[0], a01 = m[1], a02 = m[2], a10 = m[4], a11 = m[5], a12 = m[6], a20 = m[8], a21 = m[9], a22 = m[10];
  float c00 = a11 * a22 - a12 * a21, c01 = a12 * a20 - a10 * a22, c02 = a10 * a21 - a11 * a20;
  float det = a00 * c00 + a01 * c01 + a02 * c02;
  float id = 1.f / det;
  float r[3][3] = {{c00 * id, (a02 * a21 - a01 * a22) * id, (a01 * a12 - a02 * a11) * id},
                   {c01 * id, (a00 * a22 - a02 * a20) * id, (a02 * a10 - a00 * a12) * id},
                   {c02 * id, (a01 * a20 - a00 * a21) * id, (a00 * a11 - a01 * a10) * id}};
  float t[3] = {m[3], m[7], m[11]};
  float4* out = rec + 6 * (size_t)k;
  for (int row = 0; row < 3; ++row) {
    float tw = -(r[row][0] * t[0] + r[row][1] * t[1] + r[row][2] * t[2]);
    out[row] = make_float4(r[row][0], r[row][1], r[row][2], tw);
  }
  // what the traversal needs of the instance's BLAS, beside the transform
  const int4 bi = blas_info[b];
  out[3] = make_float4(blo.x, blo.y, blo.z, __int_as_float(bi.w));
  out[4] = make_float4(bhi.x, bhi.y, bhi.z, __int_as_float(bi.x));
  out[5] = make_float4(__uint_as_float(b), __uint_as_float(inst_sbt[k]), __uint_as_float(inst_id[k]),
                       __uint_as_float(inst_mask[k]));
}

__global__ void __launch_bounds__(256) k_instances(InstanceArgs A) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < A.n) instance_body(k, A);
}

// Whole two-level build of a small scene in one CTA (one launch instead of
// three): every BLAS level in turn, the instances, then the TLAS level. The
// same device routines as the separate launches, in the same order, so the
// result is the same bit for bit.
__global__ void __launch_bounds__(256) k_build_scene_small(const LevelDesc* jobs, uint32_t n_blas_jobs,
                                                            InstanceArgs A) {
  // one-leaf levels (one AABB per BLAS is common): one thread each
  for (uint32_t j = threadIdx.x; j < n_blas_jobs; j += blockDim.x)
    if (jobs[j].n == 1) single_leaf_level(jobs[j]);
  // the others with the whole CTA, one after another
  for (uint32_t j = 0; j < n_blas_jobs; ++j) {
    if (jobs[j].n > 1) {
      build_small_body(jobs[j]);
      __syncthreads();   // shared scratch reused by the next level
    }
  }
  __syncthreads();     // BLAS root boxes visible to the instance pass
  for (uint32_t k = threadIdx.x; k < A.n; k += blockDim.x) instance_body(k, A);
  __syncthreads();     // instance world boxes visible to the TLAS level
  build_small_body(jobs[n_blas_jobs]);
}

// ---- 4-wide collapse of a binary level -----------------------------------
// Every internal node at even depth becomes a 4-wide node holding its
// grandchildren (its internal children are expanded; its leaf children stay).
__global__ void __launch_bounds__(256) k_bvh2_parents(const float4* nodes, uint32_t n, uint32_t* parent) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) parent[0] = 0xFFFFFFFFu;
  if (i + 1 >= n) return;
  float4 r = nodes[4 * (size_t)i + 3];
  int a = __float_as_int(r.x), b = __float_as_int(r.y);
  if (a >= 0) parent[a] = i;
  if (b >= 0) parent[b] = i;
}

__global__ void __launch_bounds__(256) k_bvh2_even(const uint32_t* parent, uint32_t n, uint32_t* even, uint32_t* rank) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i + 1 >= n) return;
  uint32_t depth = 0;
  for (uint32_t v = i; parent[v] != 0xFFFFFFFFu; v = parent[v]) ++depth;
  uint32_t e = (depth & 1u) == 0u ? 1u : 0u;
  even[i] = e;
  rank[i] = e;
}

__global__ void __launch_bounds__(256) k_bvh4_fill(const float4* nodes, uint32_t n, const uint32_t* even,
                                                   const uint32_t* rank, float4* out) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i + 1 >= n || !even[i]) return;
  float lo[3][4], hi[3][4];
  int ref[4];
  int cnt = 0;
  const float* f = reinterpret_cast<const float*>(nodes + 4 * (size_t)i);
  for (int side = 0; side < 2; ++side) {
    int c = __float_as_int(f[12 + side]);
    if (c >= 0) {
      const float* g = reinterpret_cast<const float*>(nodes + 4 * (size_t)c);
      for (int gs = 0; gs < 2; ++gs) {
        int gr = __float_as_int(g[12 + gs]);
        for (int a = 0; a < 3; ++a) { lo[a][cnt] = g[6 * gs + a]; hi[a][cnt] = g[6 * gs + 3 + a]; }
        ref[cnt++] = gr >= 0 ? (int)rank[gr] : gr;
      }
    } else {
      for (int a = 0; a < 3; ++a) { lo[a][cnt] = f[6 * side + a]; hi[a][cnt] = f[6 * side + 3 + a]; }
      ref[cnt++] = c;
    }
  }
  for (; cnt < 4; ++cnt) {
    for (int a = 0; a < 3; ++a) { lo[a][cnt] = INFINITY; hi[a][cnt] = -INFINITY; }
    ref[cnt] = kEmptySlot;
  }
  float4* o = out + 8 * (size_t)rank[i];
  for (int a = 0; a < 3; ++a) {
    o[a] = make_float4(lo[a][0], lo[a][1], lo[a][2], lo[a][3]);
    o[3 + a] = make_float4(hi[a][0], hi[a][1], hi[a][2], hi[a][3]);
  }
  o[6] = make_float4(__int_as_float(ref[0]), __int_as_float(ref[1]), __int_as_float(ref[2]), __int_as_float(ref[3]));
  o[7] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ---- wide TLAS: greedy collapse of the binary tree --------------------------
// A wide node of width W grows from a binary node: while it has fewer than W
// children, its internal child of largest surface area (the lowest slot on
// ties) is opened into that child's two children. The internal children left
// at the end root the wide nodes below it. Which binary nodes root a wide node
// depends on the tree alone, so a prefix sum over the binary node indices
// numbers the wide nodes deterministically (the binary root is wide node 0).
// A child slot is (binary node << 1 | side): the box and reference stored on
// that side of that binary node.
constexpr uint32_t kWideEmpty = 0xFFFFFFFFu;
constexpr int kWideTopThreads = 1024;
constexpr uint32_t kWideFrontier = 4096;   // top-down pass: shared-memory frontier
constexpr uint32_t kWideDfsStart = 2048;   // frontier size at which per-root passes take over
constexpr int kWideDfsStack = 7 * 64 + 8;  // (W - 1) x the deepest traversable tree

__device__ __forceinline__ int bin_ref(const float4* nodes, uint32_t slot) {
  const float4 r = nodes[4 * (size_t)(slot >> 1) + 3];
  return __float_as_int((slot & 1u) ? r.y : r.x);
}

__device__ __forceinline__ void bin_box(const float4* nodes, uint32_t slot, float b[6]) {
  const float* f = reinterpret_cast<const float*>(nodes + 4 * (size_t)(slot >> 1)) + 6 * (slot & 1u);
  for (int k = 0; k < 6; ++k) b[k] = f[k];
}

__device__ __forceinline__ float box_half_area(const float b[6]) {
  const float dx = b[3] - b[0], dy = b[4] - b[1], dz = b[5] - b[2];
  return fmaf(dx, dy, fmaf(dy, dz, dz * dx));
}

// Grow the wide node rooted at binary node u: write its W slots, mark it a
// root (is_root and rank both 1; rank is scanned in place later) and hand
// every internal child left to push(), in slot order.
template <int W, typename Push>
__device__ void expand_wide(const float4* nodes, uint32_t u, uint32_t* slots, uint32_t* is_root, uint32_t* rank,
                            Push push) {
  // per slot: (binary node << 1 | side), the reference there and its box's area; a
  // binary node is read once, as four 16-byte loads, when it is opened
  uint32_t code[W];
  int ref[W];
  float area[W];
  auto open = [&](uint32_t p, int k0, int k1) {
    const float4* nd = nodes + 4 * (size_t)p;
    const float4 a = nd[0], b = nd[1], c = nd[2], r = nd[3];
    const float bl[6] = {a.x, a.y, a.z, a.w, b.x, b.y}, br[6] = {b.z, b.w, c.x, c.y, c.z, c.w};
    code[k0] = p << 1;
    ref[k0] = __float_as_int(r.x);
    area[k0] = box_half_area(bl);
    code[k1] = (p << 1) | 1u;
    ref[k1] = __float_as_int(r.y);
    area[k1] = box_half_area(br);
  };
  open(u, 0, 1);
  int cnt = 2;
  while (cnt < W) {
    int best = -1;
    float best_a = -1.f;
    for (int k = 0; k < cnt; ++k) {
      if (ref[k] < 0) continue;
      if (area[k] > best_a) {
        best_a = area[k];
        best = k;
      }
    }
    if (best < 0) break;
    open((uint32_t)ref[best], best, cnt);
    ++cnt;
  }
  is_root[u] = 1u;
  rank[u] = 1u;
  for (int k = 0; k < W; ++k) {
    slots[(size_t)u * W + k] = k < cnt ? code[k] : kWideEmpty;
    if (k < cnt && ref[k] >= 0) push((uint32_t)ref[k]);
  }
}

// Top of the wide tree, level by level in one block, until the frontier holds
// kWideDfsStart roots (or cannot grow inside shared memory); the frontier is
// then written out for k_wide_dfs.
template <int W>
__global__ void __launch_bounds__(kWideTopThreads) k_wide_top(const float4* nodes, uint32_t* slots, uint32_t* is_root,
                                                             uint32_t* rank, uint32_t* frontier, uint32_t* n_frontier) {
  __shared__ uint32_t buf[2][kWideFrontier];
  __shared__ uint32_t cnt[2];
  if (threadIdx.x == 0) {
    buf[0][0] = 0;
    cnt[0] = 1;
    cnt[1] = 0;
  }
  __syncthreads();
  int c = 0;
  for (;;) {
    const uint32_t m = cnt[c];
    if (m == 0 || m >= kWideDfsStart || m * (uint32_t)W > kWideFrontier) break;
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x)
      expand_wide<W>(nodes, buf[c][i], slots, is_root, rank,
                     [&](uint32_t r) { buf[c ^ 1][atomicAdd(&cnt[c ^ 1], 1u)] = r; });
    __syncthreads();
    if (threadIdx.x == 0) cnt[c] = 0;
    c ^= 1;
    __syncthreads();
  }
  const uint32_t m = cnt[c];
  for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) frontier[i] = buf[c][i];
  if (threadIdx.x == 0) *n_frontier = m;
}

// The subtree below each frontier root, depth first, one thread per root.
template <int W>
__global__ void __launch_bounds__(128) k_wide_dfs(const float4* nodes, uint32_t* slots, uint32_t* is_root,
                                                 uint32_t* rank, const uint32_t* frontier, const uint32_t* n_frontier,
                                                 uint32_t* error_word) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *n_frontier) return;
  uint32_t stack[kWideDfsStack];
  int sp = 0;
  stack[sp++] = frontier[i];
  while (sp > 0) {
    const uint32_t u = stack[--sp];
    expand_wide<W>(nodes, u, slots, is_root, rank, [&](uint32_t r) {
      if (sp < kWideDfsStack) {
        stack[sp++] = r;
      } else {   // deeper than any tree the traversal stack can take: an empty node, flagged
        is_root[r] = 1u;
        rank[r] = 1u;
        for (int k = 0; k < W; ++k) slots[(size_t)r * W + k] = kWideEmpty;
        if (error_word) atomicOr(error_word, kErrStack);
      }
    });
  }
}

// 4-wide nodes in the existing 128-byte layout.
__global__ void __launch_bounds__(256) k_wide_fill4(const float4* nodes, uint32_t n, const uint32_t* slots,
                                                    const uint32_t* is_root, const uint32_t* rank, float4* out) {
  const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u + 1 >= n || !is_root[u]) return;
  float lo[3][4], hi[3][4];
  int ref[4];
  for (int k = 0; k < 4; ++k) {
    const uint32_t sl = slots[(size_t)u * 4 + k];
    if (sl == kWideEmpty) {
      for (int a = 0; a < 3; ++a) { lo[a][k] = INFINITY; hi[a][k] = -INFINITY; }
      ref[k] = kEmptySlot;
      continue;
    }
    float b[6];
    bin_box(nodes, sl, b);
    for (int a = 0; a < 3; ++a) { lo[a][k] = b[a]; hi[a][k] = b[3 + a]; }
    const int r = bin_ref(nodes, sl);
    ref[k] = r >= 0 ? (int)rank[r] : r;
  }
  float4* o = out + 8 * (size_t)rank[u];
  for (int a = 0; a < 3; ++a) {
    o[a] = make_float4(lo[a][0], lo[a][1], lo[a][2], lo[a][3]);
    o[3 + a] = make_float4(hi[a][0], hi[a][1], hi[a][2], hi[a][3]);
  }
  o[6] = make_float4(__int_as_float(ref[0]), __int_as_float(ref[1]), __int_as_float(ref[2]), __int_as_float(ref[3]));
  o[7] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// 8-wide nodes. Float layout (224 B, 14 float4): lo.x[8], lo.y[8], lo.z[8],
// hi.x[8], hi.y[8], hi.z[8], refs[8]. Quantised layout (96 B, 6 float4), after
// Ylitie et al. 2017: origin.xyz and three biased power-of-two exponents, then
// per axis the 8 lower and 8 upper child bounds as bytes (lo[0..3], lo[4..7],
// hi[0..3], hi[4..7] words), then refs[8]. A child bound decodes to
// origin + q * 2^e. Quantisation is conservative with a margin of one step on
// either side (the origin sits one step below the node), so a decoded box
// contains the float box by at least one step; the step is at least 2^-18 of
// the node's coordinate magnitude, so the margin exceeds the rounding of the
// slab tests and the decoded boxes pass every ray the float boxes pass.
template <bool kQuant>
__global__ void __launch_bounds__(256) k_wide_fill8(const float4* nodes, uint32_t n, const uint32_t* slots,
                                                    const uint32_t* is_root, const uint32_t* rank, float4* out) {
  const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u + 1 >= n || !is_root[u]) return;
  float lo[3][8], hi[3][8];
  int ref[8];
  for (int k = 0; k < 8; ++k) {
    const uint32_t sl = slots[(size_t)u * 8 + k];
    if (sl == kWideEmpty) {
      for (int a = 0; a < 3; ++a) { lo[a][k] = INFINITY; hi[a][k] = -INFINITY; }
      ref[k] = kEmptySlot;
      continue;
    }
    float b[6];
    bin_box(nodes, sl, b);
    for (int a = 0; a < 3; ++a) { lo[a][k] = b[a]; hi[a][k] = b[3 + a]; }
    const int r = bin_ref(nodes, sl);
    ref[k] = r >= 0 ? (int)rank[r] : r;
  }
  if (!kQuant) {
    float4* o = out + 14 * (size_t)rank[u];
    for (int a = 0; a < 3; ++a) {
      o[2 * a] = make_float4(lo[a][0], lo[a][1], lo[a][2], lo[a][3]);
      o[2 * a + 1] = make_float4(lo[a][4], lo[a][5], lo[a][6], lo[a][7]);
      o[6 + 2 * a] = make_float4(hi[a][0], hi[a][1], hi[a][2], hi[a][3]);
      o[6 + 2 * a + 1] = make_float4(hi[a][4], hi[a][5], hi[a][6], hi[a][7]);
    }
    o[12] = make_float4(__int_as_float(ref[0]), __int_as_float(ref[1]), __int_as_float(ref[2]), __int_as_float(ref[3]));
    o[13] = make_float4(__int_as_float(ref[4]), __int_as_float(ref[5]), __int_as_float(ref[6]), __int_as_float(ref[7]));
    return;
  }
  float org[3];
  uint32_t ebits = 0, w[3][4];
  for (int a = 0; a < 3; ++a) {
    float L = INFINITY, H = -INFINITY;
    for (int k = 0; k < 8; ++k)
      if (ref[k] != kEmptySlot) {
        L = fminf(L, lo[a][k]);
        H = fmaxf(H, hi[a][k]);
      }
    // step 2^e: at least 1/248 of the extent and 2^-18 of the magnitude
    const double need = fmax(((double)H - (double)L) / 248.0, ldexp(fmax(fabs((double)L), fabs((double)H)), -18));
    int e;
    frexp(need > 0.0 ? need : 1e-30, &e);   // need < 2^e
    e = max(-126, min(127, e));
    const double step = ldexp(1.0, e);
    org[a] = __double2float_rd((double)L - step);
    w[a][0] = w[a][1] = w[a][2] = w[a][3] = 0;
    for (int k = 0; k < 8; ++k) {
      uint32_t ql = 0, qh = 0;
      if (ref[k] != kEmptySlot) {
        const double fl = floor(((double)lo[a][k] - (double)org[a]) / step) - 1.0;
        const double fh = ceil(((double)hi[a][k] - (double)org[a]) / step) + 1.0;
        ql = (uint32_t)fmin(fmax(fl, 0.0), 255.0);
        qh = (uint32_t)fmin(fmax(fh, 0.0), 255.0);
      }
      w[a][k >> 2] |= ql << (8 * (k & 3));
      w[a][2 + (k >> 2)] |= qh << (8 * (k & 3));
    }
    ebits |= (uint32_t)(e + 127) << (8 * a);
  }
  float4* o = out + 6 * (size_t)rank[u];
  o[0] = make_float4(org[0], org[1], org[2], __uint_as_float(ebits));
  for (int a = 0; a < 3; ++a)
    o[1 + a] = make_float4(__uint_as_float(w[a][0]), __uint_as_float(w[a][1]), __uint_as_float(w[a][2]),
                           __uint_as_float(w[a][3]));
  o[4] = make_float4(__int_as_float(ref[0]), __int_as_float(ref[1]), __int_as_float(ref[2]), __int_as_float(ref[3]));
  o[5] = make_float4(__int_as_float(ref[4]), __int_as_float(ref[5]), __int_as_float(ref[6]), __int_as_float(ref[7]));
}

// Zero-fill by a kernel instead of cudaMemsetAsync: a memset may run on a copy
// engine, where it queues behind a large device-to-host copy of another stream
// (the pipelined readback of earlier images) and stalls the build.
__global__ void __launch_bounds__(256) k_zero_u32(uint32_t* a, uint32_t* b, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    a[i] = 0u;
    if (b) b[i] = 0u;
  }
}

// Vertex bounds of each triangle (exact: min/max only).
__global__ void __launch_bounds__(256) k_tri_boxes(const float* v, const uint32_t* idx, uint32_t n, float* boxes) {
  uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const uint32_t a = idx[3 * (size_t)t], b = idx[3 * (size_t)t + 1], c = idx[3 * (size_t)t + 2];
  for (int k = 0; k < 3; ++k) {
    float x = v[3 * (size_t)a + k], y = v[3 * (size_t)b + k], z = v[3 * (size_t)c + k];
    boxes[6 * (size_t)t + k] = fminf(fminf(x, y), z);
    boxes[6 * (size_t)t + 3 + k] = fmaxf(fmaxf(x, y), z);
  }
}

}  // namespace

int launch_triangle_boxes(const float* vertices, const uint32_t* indices, uint32_t n_tri, float* boxes,
                          cudaStream_t s) {
  if (n_tri == 0) return 0;
  k_tri_boxes<<<(n_tri + 255) / 256, 256, 0, s>>>(vertices, indices, n_tri, boxes);
  return 1;
}

int launch_collapse4(const float4* nodes2, uint32_t n, uint32_t* parent, uint32_t* even, uint32_t* rank,
                     float4* nodes4, cudaStream_t s) {
  if (n < 2) return 0;
  uint32_t nb = (n + 255) / 256;
  k_bvh2_parents<<<nb, 256, 0, s>>>(nodes2, n, parent);
  k_bvh2_even<<<nb, 256, 0, s>>>(parent, n, even, rank);
  k_radix_scan<<<1, 1024, 0, s>>>(rank, n - 1);            // exclusive prefix sum: 4-wide node index
  k_bvh4_fill<<<nb, 256, 0, s>>>(nodes2, n, even, rank, nodes4);
  return 4;
}

namespace {
void zero_u32(uint32_t* a, uint32_t* b, uint32_t n, cudaStream_t s) {
  if (n == 0) return;
  const uint32_t blocks = std::min<uint32_t>((n + 255) / 256, 1184u);
  k_zero_u32<<<blocks, 256, 0, s>>>(a, b, n);
}
}  // namespace

int launch_collapse_wide(const float4* nodes2, uint32_t n, int format, const WideScratch& ws, float4* out,
                         uint32_t* error_word, cudaStream_t s) {
  if (n < 2) return 0;
  const uint32_t nb = (n + 255) / 256;
  const int W = format == kWide4 ? 4 : 8;
  zero_u32(ws.is_root, ws.rank, n - 1, s);
  const uint32_t dfs_blocks = (kWideFrontier + 127) / 128;
  if (W == 4) {
    k_wide_top<4><<<1, kWideTopThreads, 0, s>>>(nodes2, ws.slots, ws.is_root, ws.rank, ws.frontier, ws.n_frontier);
    k_wide_dfs<4><<<dfs_blocks, 128, 0, s>>>(nodes2, ws.slots, ws.is_root, ws.rank, ws.frontier, ws.n_frontier,
                                             error_word);
  } else {
    k_wide_top<8><<<1, kWideTopThreads, 0, s>>>(nodes2, ws.slots, ws.is_root, ws.rank, ws.frontier, ws.n_frontier);
    k_wide_dfs<8><<<dfs_blocks, 128, 0, s>>>(nodes2, ws.slots, ws.is_root, ws.rank, ws.frontier, ws.n_frontier,
                                             error_word);
  }
  k_radix_scan<<<1, 1024, 0, s>>>(ws.rank, n - 1);   // exclusive prefix sum: wide node index
  if (format == kWide4) k_wide_fill4<<<nb, 256, 0, s>>>(nodes2, n, ws.slots, ws.is_root, ws.rank, out);
  else if (format == kWide8) k_wide_fill8<false><<<nb, 256, 0, s>>>(nodes2, n, ws.slots, ws.is_root, ws.rank, out);
  else k_wide_fill8<true><<<nb, 256, 0, s>>>(nodes2, n, ws.slots, ws.is_root, ws.rank, out);
  return 5;
}

int launch_build_small(const LevelDesc* d_jobs, uint32_t n_jobs, cudaStream_t s) {
  if (n_jobs == 0) return 0;
  k_build_small<<<n_jobs, 256, 0, s>>>(d_jobs);
  return 1;
}

int launch_build_small_one(const LevelDesc& J, cudaStream_t s) {
  if (J.n == 0) return 0;
  k_build_small_one<<<1, 256, 0, s>>>(J);
  return 1;
}

int launch_build_large(const LevelDesc& J, const BuildScratch& sc, cudaStream_t s) {
  const uint32_t n = J.n;
  int launches = 0;
  uint32_t nb = (n + 255) / 256;
  uint32_t n_partial = nb < kMaxPartials ? nb : kMaxPartials;
  k_centroid_partial<<<n_partial, 256, 0, s>>>(J, sc.partial);
  uint32_t nb_m = nb < 2048u ? nb : 2048u;
  k_morton<<<nb_m, 256, 0, s>>>(J, sc.partial, (int)n_partial, sc.keys[0], sc.vals[0]);
  launches += 2;
  const uint32_t tiles = sort_tiles(n);
  int cur = 0;
  for (int pass = 0; pass < 4; ++pass) {
    int shift = 8 * pass;
    k_radix_hist<<<tiles, 256, 0, s>>>(sc.keys[cur], n, shift, sc.hist, tiles);
    k_radix_scan<<<1, 1024, 0, s>>>(sc.hist, 256 * tiles);
    k_radix_scatter<<<tiles, 256, 0, s>>>(sc.keys[cur], sc.vals[cur], sc.keys[1 - cur], sc.vals[1 - cur], n, shift,
                                          sc.hist, tiles);
    cur = 1 - cur;
    launches += 3;
  }
  zero_u32(sc.counters, nullptr, n - 1, s);
  k_karras<<<nb, 256, 0, s>>>(J, sc.keys[cur], sc.vals[cur], sc.parent_int, sc.parent_leaf, nullptr);
  k_refit<<<nb, 256, 0, s>>>(J, sc.vals[cur], sc.parent_int, sc.parent_leaf, sc.counters, nullptr);
  launches += 3;
  return launches;
}

int launch_build_ploc(const LevelDesc& J, const BuildScratch& sc, uint32_t* error_word, cudaStream_t s,
                      cudaEvent_t after, cudaEvent_t mark) {
  const uint32_t n = J.n;
  if (n < 2) return launch_build_large(J, sc, s);
  int launches = 0;
  // Morton order of the leaves: the LBVH's centroid bounds, codes and radix sort
  uint32_t nb = (n + 255) / 256;
  uint32_t n_partial = nb < kMaxPartials ? nb : kMaxPartials;
  k_centroid_partial<<<n_partial, 256, 0, s>>>(J, sc.partial);
  uint32_t nb_m = nb < 2048u ? nb : 2048u;
  k_morton<<<nb_m, 256, 0, s>>>(J, sc.partial, (int)n_partial, sc.keys[0], sc.vals[0]);
  launches += 2;
  const uint32_t tiles = sort_tiles(n);
  int cur = 0;
  for (int pass = 0; pass < 4; ++pass) {
    int shift = 8 * pass;
    k_radix_hist<<<tiles, 256, 0, s>>>(sc.keys[cur], n, shift, sc.hist, tiles);
    k_radix_scan<<<1, 1024, 0, s>>>(sc.hist, 256 * tiles);
    k_radix_scatter<<<tiles, 256, 0, s>>>(sc.keys[cur], sc.vals[cur], sc.keys[1 - cur], sc.vals[1 - cur], n, shift,
                                          sc.hist, tiles);
    cur = 1 - cur;
    launches += 3;
  }
  // Clustering in one cooperative launch. Scratch: the histogram's buffer holds
  // the header and the per-block counts, the refit counters the nearest
  // neighbours, and the wide TLAS buffer (written only by the collapse that
  // follows the clustering) the two lists of cluster records.
  if (cudaFuncSetAttribute(k_ploc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPlocSmem) != cudaSuccess)
    return -1;
  static int blocks_per_sm = 0, n_sm = 0;
  if (!blocks_per_sm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_ploc, kPlocThreads, kPlocSmem);
    if (blocks_per_sm > 1) blocks_per_sm = 1;   // one block per SM: cheaper grid barriers
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  const size_t hist_bytes = sizeof(uint32_t) * 256 * (size_t)tiles;
  uint32_t grid = (uint32_t)(blocks_per_sm * n_sm);
  grid = std::min(grid, (n + kPlocThreads - 1) / kPlocThreads);
  grid = std::min(grid, (uint32_t)((hist_bytes - kPlocPartOffset) / sizeof(unsigned long long)));
  grid = std::max(grid, 1u);
  PlocArgs A;
  A.J = J;
  A.codes = sc.keys[cur];
  A.vals = sc.vals[cur];
  A.R[0] = reinterpret_cast<float4*>(sc.cluster_boxes);
  A.R[1] = A.R[0] + 2 * (size_t)n;
  A.nn = reinterpret_cast<int*>(sc.counters);
  A.hdr = sc.hist;
  A.error_word = error_word;
  A.part = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(sc.hist) + kPlocPartOffset);
  zero_u32(sc.hist, nullptr, (uint32_t)(kPlocPartOffset / sizeof(uint32_t)), s);
  ++launches;
  void* args[] = {&A};
  if (after && cudaStreamWaitEvent(s, after, 0) != cudaSuccess) return -1;
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_ploc, dim3(grid), dim3(kPlocThreads), args, kPlocSmem, s);
  if (e != cudaSuccess) return -1;
  if (mark && cudaEventRecord(mark, s) != cudaSuccess) return -1;
  ++launches;
  // the LBVH's tree passes, which return at once unless a barrier of the
  // clustering gave up
  const uint32_t* done = sc.hist + kHdrOk;
  zero_u32(sc.counters, nullptr, n - 1, s);
  k_karras<<<nb, 256, 0, s>>>(J, sc.keys[cur], sc.vals[cur], sc.parent_int, sc.parent_leaf, done);
  k_refit<<<nb, 256, 0, s>>>(J, sc.vals[cur], sc.parent_int, sc.parent_leaf, sc.counters, done);
  return launches + 3;
}

int launch_instances(const InstanceArgs& A, cudaStream_t s) {
  if (A.n == 0) return 0;
  k_instances<<<(A.n + 255) / 256, 256, 0, s>>>(A);
  return 1;
}

int launch_build_scene_small(const LevelDesc* d_jobs, uint32_t n_blas_jobs, const InstanceArgs& A, cudaStream_t s) {
  k_build_scene_small<<<1, 256, 0, s>>>(d_jobs, n_blas_jobs, A);
  return 1;
}

}  // namespace pr
