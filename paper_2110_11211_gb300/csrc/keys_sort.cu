// Hilbert keys of the grid points and their sort into curve order.
//
// Sec. 3.2 / Sec. 3.3: the points are mapped by the inverse discrete Hilbert
// curve s_n^{-1} at the finest resolution n = max_j l_j; the paper builds on
// Skilling's construction ("Programming the Hilbert curve", 2004).  Point k is
// placed at cell X_j = k_j 2^{n - l_j}; Skilling's axes-to-transpose transform
// gives the key's bits level by level, axis 0 first.  Algorithm 1, step 3 sorts
// the points by key: an LSD radix sort with 8-bit digits over the d*n key bits.
#include "sfcdd_internal.cuh"

namespace sfcdd {

// One thread per lexicographic id; D is the dimension (compile time so the
// per-axis arrays stay in registers).
template <int D>
__global__ void k_keygen(GridDev g, unsigned long long* __restrict__ keys,
                         unsigned* __restrict__ codes) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  unsigned code;
  keys[id] = hilbert_key_of<D>(g, id, code);
  codes[id] = code;
}

void launch_keygen(const GridDev& g, unsigned long long* keys, unsigned* codes, cudaStream_t s) {
  const int bs = 256, nb = (g.N + bs - 1) / bs;
  switch (g.d) {
    case 1: k_keygen<1><<<nb, bs, 0, s>>>(g, keys, codes); break;
    case 2: k_keygen<2><<<nb, bs, 0, s>>>(g, keys, codes); break;
    case 3: k_keygen<3><<<nb, bs, 0, s>>>(g, keys, codes); break;
    case 4: k_keygen<4><<<nb, bs, 0, s>>>(g, keys, codes); break;
    case 5: k_keygen<5><<<nb, bs, 0, s>>>(g, keys, codes); break;
    case 6: k_keygen<6><<<nb, bs, 0, s>>>(g, keys, codes); break;
    case 7: k_keygen<7><<<nb, bs, 0, s>>>(g, keys, codes); break;
    default: k_keygen<8><<<nb, bs, 0, s>>>(g, keys, codes); break;
  }
}

// ---------------------------------------------------------------------------
// LSD radix sort of (uint64 key, uint32 value) pairs, 8-bit digits, stable.
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;
constexpr int RS_WARPS = RS_THREADS / 32;

__global__ void k_rs_hist(const unsigned long long* __restrict__ keys, int n, int shift,
                          unsigned* __restrict__ hist, int nblocks) {
  __shared__ unsigned h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int base = blockIdx.x * RS_TILE;
  for (int k = threadIdx.x; k < RS_TILE; k += RS_THREADS) {
    const int i = base + k;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of `len` counts in place, one block of 1024 threads.
__global__ void k_rs_scan(unsigned* __restrict__ a, int len) {
  __shared__ unsigned warp_tot[32];
  __shared__ unsigned carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int base = 0; base < len; base += 1024) {
    const int i = base + threadIdx.x;
    const unsigned v = i < len ? a[i] : 0u;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
      unsigned t = warp_tot[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    const unsigned before = (w > 0 ? warp_tot[w - 1] : 0u) + carry;
    if (i < len) a[i] = before + x - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry = before + x;
    __syncthreads();
  }
}

__global__ void k_rs_scatter(const unsigned long long* __restrict__ kin,
                             const unsigned* __restrict__ vin, unsigned long long* __restrict__ kout,
                             unsigned* __restrict__ vout, int n, int shift,
                             const unsigned* __restrict__ offs, int nblocks) {
  __shared__ unsigned base[256];
  __shared__ unsigned wcnt[RS_WARPS][257];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  base[tid] = offs[tid * nblocks + blockIdx.x];
  const unsigned lt = (1u << lane) - 1u;
  for (int round = 0; round < RS_ROUNDS; ++round) {
    const int i = blockIdx.x * RS_TILE + round * RS_THREADS + tid;
    const bool valid = i < n;
    unsigned long long key = 0;
    unsigned val = 0;
    int digit = 256;  // sentinel bucket for the ragged tail
    if (valid) {
      key = kin[i];
      val = vin[i];
      digit = (int)((key >> shift) & 255u);
    }
    for (int k = tid; k < RS_WARPS * 257; k += RS_THREADS) (&wcnt[0][0])[k] = 0;
    __syncthreads();
    const unsigned peers = __match_any_sync(0xffffffffu, digit);
    const unsigned rank = __popc(peers & lt);
    if (rank == 0) wcnt[w][digit] = __popc(peers);
    __syncthreads();
    unsigned pos = 0;
    if (valid) {
      unsigned before = 0;
      for (int ww = 0; ww < w; ++ww) before += wcnt[ww][digit];
      pos = base[digit] + before + rank;
    }
    __syncthreads();
    {
      unsigned tot = 0;
#pragma unroll
      for (int ww = 0; ww < RS_WARPS; ++ww) tot += wcnt[ww][tid];
      base[tid] += tot;
    }
    if (valid) {
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
  }
}

size_t radix_sort_temp_bytes(int n) {
  const int nblocks = (n + RS_TILE - 1) / RS_TILE;
  return (size_t)n * (sizeof(unsigned long long) + sizeof(unsigned)) +
         (size_t)256 * nblocks * sizeof(unsigned) + 256;
}

// Sorts keys/vals in place (ping-pong through temp); `bits` significant key bits.
void radix_sort_pairs(unsigned long long* keys, unsigned* vals, int n, int bits, void* temp,
                      cudaStream_t s, int* launches) {
  if (n <= 1) return;
  const int nblocks = (n + RS_TILE - 1) / RS_TILE;
  unsigned long long* k2 = reinterpret_cast<unsigned long long*>(temp);
  unsigned* v2 = reinterpret_cast<unsigned*>(k2 + n);
  unsigned* hist = v2 + n;
  hist = reinterpret_cast<unsigned*>((reinterpret_cast<uintptr_t>(hist) + 15) & ~uintptr_t(15));
  const int passes = (bits + 7) / 8;
  unsigned long long *ka = keys, *kb = k2;
  unsigned *va = vals, *vb = v2;
  for (int ps = 0; ps < passes; ++ps) {
    const int shift = ps * 8;
    k_rs_hist<<<nblocks, RS_THREADS, 0, s>>>(ka, n, shift, hist, nblocks);
    k_rs_scan<<<1, 1024, 0, s>>>(hist, 256 * nblocks);
    k_rs_scatter<<<nblocks, RS_THREADS, 0, s>>>(ka, va, kb, vb, n, shift, hist, nblocks);
    if (launches) *launches += 3;
    unsigned long long* tk = ka; ka = kb; kb = tk;
    unsigned* tv = va; va = vb; vb = tv;
  }
  if (ka != keys) {
    cudaMemcpyAsync(keys, ka, (size_t)n * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(vals, va, (size_t)n * sizeof(unsigned), cudaMemcpyDeviceToDevice, s);
  }
}

__global__ void k_invpad_fill(const unsigned* __restrict__ code, int* __restrict__ invpad, int n) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) invpad[code[p]] = p;
}

void launch_invpad_fill(const unsigned* curve_code, int* invpad, int n, cudaStream_t s) {
  k_invpad_fill<<<(n + 255) / 256, 256, 0, s>>>(curve_code, invpad, n);
}

__global__ void k_perm_lex(GridDev g, const unsigned* __restrict__ code, int* __restrict__ perm) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.N) return;
  const unsigned c = code[p];
  int id = 0;
  for (int j = 0; j < g.d; ++j) {
    const int kj = (int)((c >> g.off[j]) & ((1u << g.lev[j]) - 1u));
    id += (kj - 1) * g.stride[j];
  }
  perm[p] = id;
}

void launch_perm_lex(const GridDev& g, const unsigned* curve_code, int* perm, cudaStream_t s) {
  k_perm_lex<<<(g.N + 255) / 256, 256, 0, s>>>(g, curve_code, perm);
}

}  // namespace sfcdd
