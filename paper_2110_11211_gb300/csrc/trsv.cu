// Batched forward / backward substitution with the Cholesky factors of the
// local matrices A_i and of the coarse matrix A_0 (Algorithm 2, steps 2-3: the
// factorization is done once in the setup phase and every application of the
// preconditioner only runs the two triangular solves, Sec. 3.1).
//
// Factor form.  With D = blockdiag(D_J), D_J the lower block-triangular
// diagonal block of cb x cb tiles (cb = 1 for the local factors, 4 for the
// coarse one), the setup splits L = Lh D with Lh = L D^{-1} (identity diagonal
// blocks), so that A = Lh (D D^T) Lh^T and, for tile rows I in block J,
//   forward   z_I = b_I - sum_{K < first row of J} Lh_IK z_K
//   backward  x_I = sum_{K in J} E_J(I, K) z_K - sum_{K after J} Lh_KI^T x_K,
// E_J = D_J^{-T} D_J^{-1}.  The forward reads the Lh tiles (row-major); the
// backward reads a second copy holding Lh_KI^T in slot (K, I), and the E tiles
// in the block's own slots (lower ones in that copy, upper ones in the first
// array, where Lh is the identity).  Both sweeps stream contiguous row slabs;
// all rows of a block depend only on earlier blocks, so the row-to-row chain
// has nt / cb steps, each carrying the GEMVs with the previous block's tiles.
//
// Parallel layout: one CTA per work item (matrix, tile row, slab), a slab
// being R = 64 / S consecutive rows of the tile row (S = 1, 2 or 4 per matrix:
// splitting the rows of a long chain spreads its FP64 GEMVs over S SMs).  CTAs
// take tickets from a monotone counter and map them through a work list in
// which every item comes after the items it depends on, so a CTA only ever
// waits for CTAs that already started (no deadlock, whatever the residency).
// Row results are their own ready flags: before a launch the result slots hold
// a sentinel NaN bit pattern, every slot is written exactly once per launch
// with a relaxed store, and a consumer polls the slots it needs with relaxed
// loads until none holds the sentinel (bounded spin; a timeout sets the error
// word and the CTA still drains its copies before it returns).  Only consumer
// warp 0 polls; it hands the 64 values of each dependency to the other warps
// through shared memory and a per-stage mbarrier, so one straggling lane
// cannot hold up eight warps and the L2 sees one poller per CTA.  The forward
// launch resets the backward slots of its slab and also writes its results to
// a plain buffer zc; the backward launch reads z from zc and resets the forward
// slots of its slab (nothing reads them during the backward launch).
//
// Data movement: a producer warp streams the item's tile slabs (E tiles first
// in the backward) from HBM into a shared-memory ring with bulk asynchronous
// copies (cp.async.bulk, completion on mbarriers); eight consumer warps wait on
// the ring's mbarriers, apply the slabs, and free the stages.  The ring holds
// two tiles of the launch's local precision (FP64 64 KB, FP32 32 KB, BF16
// 16 KB), so low-precision launches keep more CTAs resident; coarse items of
// such launches run in 16-row slabs (8 KB stages).
#include "sfcdd_internal.cuh"

namespace sfcdd {

constexpr int NCONS = 256;                 // consumer threads: 8 warps
constexpr int NTHR = NCONS + 32;           // + one producer warp
constexpr int MAXST = 8;
constexpr long long SPIN_LIMIT = 1ll << 22;
constexpr long long MBAR_LIMIT = 1ll << 26;
constexpr long long SPIN_FAST = 1 << 12;   // polls before the poller starts to back off

// Shared-memory plan of a launch whose local factors have element size ES.
template <int ES>
struct Plan {
  // slab ring: 32 KB (one FP64 or two FP32 tiles, four BF16), so that four or more
  // CTAs fit an SM; a 64-row FP64 slab then has a single stage
  static constexpr int RING = (ES == 8 ? 1 : 2) * TILE2 * ES;
  static constexpr int ZBUF = MAXST * TILE * 8;
  static constexpr int BYTES = RING + ZBUF + 3 * MAXST * 8;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for a phase of an mbarrier; records TIMEOUT (site) if it gives up.
__device__ __forceinline__ void mbar_wait(unsigned long long* bar, unsigned parity, ErrWord* err,
                                          int site) {
  long long it = 0;
  while (!mbar_try_wait(bar, parity)) {
    if (++it > MBAR_LIMIT) {
      if (atomicCAS(&err->code, 0, (int)SFCDD_ERR_TIMEOUT) == 0) err->index = site;
      return;
    }
  }
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes,
                                          unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ double2 ld_relaxed2(const double* p) {
  unsigned long long a, b;
  asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
  return make_double2(__longlong_as_double((long long)a), __longlong_as_double((long long)b));
}
__device__ __forceinline__ void st_relaxed(double* p, double v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(__double_as_longlong(v))
               : "memory");
}
__device__ __forceinline__ bool is_pending(double v) {
  return (unsigned long long)__double_as_longlong(v) == TRSV_PENDING;
}
// Polls two consecutive result slots (16-byte aligned) until both hold values
// (bounded; a timeout records TIMEOUT and returns whatever is there).
__device__ __forceinline__ double2 wait_pair(const double* p, ErrWord* err, int site) {
  double2 v = ld_relaxed2(p);
  long long it = 0;
  while (is_pending(v.x) || is_pending(v.y)) {
    if (++it > SPIN_FAST) __nanosleep(64);
    if ((it & 1023) == 0 &&
        (*((volatile int*)&err->code) != 0 || it > SPIN_LIMIT)) {
      if (atomicCAS(&err->code, 0, (int)SFCDD_ERR_TIMEOUT) == 0) err->index = site;
      break;
    }
    v = ld_relaxed2(p);
  }
  return v;
}

// Two consecutive elements of a shared-memory slab row as the accumulation type.
__device__ __forceinline__ void sm_pair(const double* p, double& a, double& b) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  a = v.x;
  b = v.y;
}
__device__ __forceinline__ void sm_pair(const float* p, float& a, float& b) {
  const float2 v = *reinterpret_cast<const float2*>(p);
  a = v.x;
  b = v.y;
}
__device__ __forceinline__ void sm_pair(const __nv_bfloat16* p, float& a, float& b) {
  const unsigned u = *reinterpret_cast<const unsigned*>(p);
  a = __uint_as_float(u << 16);
  b = __uint_as_float(u & 0xffff0000u);
}

// Sums v[i] over the 32 lanes for the warp's RPW rows: log2(RPW) halving
// exchanges (each lane keeps the half its lane bit selects) followed by a
// butterfly over the remaining lanes.  Every lane returns the total of row
// `row`; the 32 / RPW lanes of a group hold the same row.
template <int RPW, class A>
__device__ __forceinline__ A reduce_rows(A (&v)[RPW], int& row) {
  const int lane = threadIdx.x & 31;
  A cur[RPW];
#pragma unroll
  for (int i = 0; i < RPW; ++i) cur[i] = v[i];
  row = 0;
  int dist = 16;
#pragma unroll
  for (int width = RPW; width > 1; width >>= 1) {
    const bool hi = (lane & dist) != 0;
#pragma unroll
    for (int i = 0; i < width / 2; ++i) {
      const A keep = hi ? cur[i + width / 2] : cur[i];
      const A send = hi ? cur[i] : cur[i + width / 2];
      cur[i] = keep + __shfl_xor_sync(0xffffffffu, send, dist);
    }
    row = 2 * row + (hi ? 1 : 0);
    dist >>= 1;
  }
  A t = cur[0];
#pragma unroll
  for (; dist >= 1; dist >>= 1) t += __shfl_xor_sync(0xffffffffu, t, dist);
  return t;
}

struct RowSmem {
  unsigned char* ring;
  double* zbuf;               // [MAXST][TILE] dependency values of each stage
  unsigned long long* full;   // [MAXST]
  unsigned long long* empty;  // [MAXST]
  unsigned long long* zbar;   // [MAXST] zbuf of the stage is filled
};

// One work item: rows [R s, R s + R) of tile row r of matrix m.
//   FWD: z_r = b_r - sum_{c<r} Lh_rc z_c          (tiles lt, row list)
//   BWD: x_r = E_r z_r - sum_{c>r} Lh_cr^T x_c     (tiles ut, column list)
template <class T, class A, int R, bool FWD, int RING>
__device__ void sweep_item(const TrsvArgs& a, const T* __restrict__ lt, const T* __restrict__ ut,
                           int m, int r, int slab, int cb, const RowSmem& sm) {
  constexpr int RPW = R / 8;                        // rows per consumer warp
  constexpr unsigned SB = R * TILE * sizeof(T);     // slab bytes
  constexpr int NS = (RING / (int)SB) < MAXST ? (RING / (int)SB) : MAXST;
  static_assert(NS >= 1, "slab larger than the ring");
  const long long tb = a.ts.tbase[m];
  const int vb = a.ts.vbase[m];
  const int fb = vb / TILE;
  const long long soff = (long long)R * slab * TILE;  // slab offset inside a tile
  // r's unit diagonal block: tile rows [blk0, blk1)
  const int blk0 = r / cb * cb;
  const int blk1 = min(blk0 + cb, a.ts.nt[m]);
  // tile t of the item: forward, Lh (r, k0 + t) against z of row k0 + t, the
  // tiles left of the block; backward, first the nE tiles E(r, blk0 + t)
  // against z (from zc), then Lh^T (c, r) for the rows c below the block (from
  // the last) against x_c
  int ntile, nE = 0, ncl = 0, k0 = 0;
  const int* cl = nullptr;
  const T* row0 = nullptr;
  if (FWD) {
    k0 = a.ts.kmin[fb + r];
    row0 = lt + tb + (long long)a.ts.rowoff[fb + r] * TILE2 + soff;  // tile (r, k0)
    ntile = blk0 > k0 ? blk0 - k0 : 0;
  } else {
    cl = a.ts.colidx + a.ts.colptr[fb + r];  // rows c > r reaching column r, ascending
    ncl = a.ts.colptr[fb + r + 1] - a.ts.colptr[fb + r];
    int skip = 0;
    while (skip < ncl && cl[skip] < blk1) ++skip;  // rows of r's own block
    cl += skip;
    ncl -= skip;
    nE = blk1 - blk0;
    ntile = nE + ncl;
  }
  if (threadIdx.x >= NCONS) {
    if (threadIdx.x == NCONS) {
      for (int t = 0; t < ntile; ++t) {
        const int s = t % NS, k = t / NS;
        if (k >= 1) mbar_wait(&sm.empty[s], (k - 1) & 1, a.err, 10);
        const T* src;
        if (FWD) {
          src = row0 + (long long)t * TILE2;
        } else if (t < nE) {
          // E(r, kp): ut holds the block's lower tiles, the tiles array its upper ones
          const int kp = blk0 + t;
          src = (kp <= r ? ut + tile_at(a.ts, tb, fb, r, kp) : lt + tile_at(a.ts, tb, fb, kp, r)) +
                soff;
        } else {
          src = ut + tile_at(a.ts, tb, fb, cl[ncl - 1 - (t - nE)], r) + soff;
        }
        mbar_expect_tx(&sm.full[s], SB);
        bulk_copy(sm.ring + (size_t)s * SB, src, SB, &sm.full[s]);
      }
    }
    return;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int rloc = RPW * w;                 // first slab row of this warp
  const int rbase = r * TILE + R * slab;    // first row of the slab in the matrix
  A acc[RPW];
#pragma unroll
  for (int i = 0; i < RPW; ++i) acc[i] = A(0);
  double bval = 0.0;
  if (FWD) {
    // right-hand side of this warp's rows (lane i < RPW holds row rloc + i)
    if (lane < RPW) {
      const int grow = rbase + rloc + lane;
      if (grow < a.ts.n[m]) {
        const MatDesc md = a.md[m];
        if (md.coarse) {
          bval = a.g0[md.rhs_base + (a.cblock ? a.cblock[grow] : grow)];
        } else {
          int pos;
          if (a.ts.lperm) {
            pos = a.ts.lperm[vb + grow];
          } else {
            pos = md.start + grow;
            if (pos >= md.rhs_len) pos -= md.rhs_len;
          }
          bval = a.rhs[md.rhs_base + pos];
        }
      }
    }
    // the backward slots of this slab are reset here (nobody reads them in this launch)
    if (threadIdx.x < R)
      a.dout[vb + rbase + threadIdx.x] = __longlong_as_double((long long)TRSV_PENDING);
  } else {
    // the forward slots of this slab are reset for the next forward launch
    if (threadIdx.x < R)
      a.y[vb + rbase + threadIdx.x] = __longlong_as_double((long long)TRSV_PENDING);
  }
  for (int t = 0; t < ntile; ++t) {
    const int s = t % NS;
    const unsigned ph = (t / NS) & 1;
    double* zs = sm.zbuf + s * TILE;
    double2 v;
    if (w == 0) {
      // every warp is done with the previous use of stage s (and of zs)
      if (t >= NS) mbar_wait(&sm.empty[s], ph ^ 1, a.err, 13);
      // z of the block comes from the forward launch (a previous kernel, never
      // the sentinel), the other vectors from this launch
      const double* dp = FWD      ? a.y + vb + (k0 + t) * TILE
                         : t < nE ? a.zc + vb + (blk0 + t) * TILE
                                  : a.dout + vb + cl[ncl - 1 - (t - nE)] * TILE;
      v = wait_pair(dp + 2 * lane, a.err, FWD ? 1 : 2);
      *reinterpret_cast<double2*>(zs + 2 * lane) = v;
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.zbar[s]);
    } else {
      mbar_wait(&sm.zbar[s], ph, a.err, 14);
      v = *reinterpret_cast<const double2*>(zs + 2 * lane);
    }
    // backward: + E z, - Lh^T x
    const bool neg = !FWD && t >= nE;
    const A v0 = A(neg ? -v.x : v.x), v1 = A(neg ? -v.y : v.y);
    mbar_wait(&sm.full[s], ph, a.err, 11);
    const T* st = reinterpret_cast<const T*>(sm.ring + (size_t)s * SB);
#pragma unroll
    for (int i = 0; i < RPW; ++i) {
      A l0, l1;
      sm_pair(st + (rloc + i) * TILE + 2 * lane, l0, l1);
      acc[i] = fma(l0, v0, acc[i]);
      acc[i] = fma(l1, v1, acc[i]);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.empty[s]);
  }
  int row;
  const A tot = reduce_rows<RPW>(acc, row);
  const int orow = vb + rbase + rloc + row;
  if (FWD) {
    const double br = __shfl_sync(0xffffffffu, bval, row);  // row i's rhs sits in lane i
    if ((lane & (32 / RPW - 1)) == 0) {
      const double zv = double(A(br) - tot);
      st_relaxed(a.y + orow, zv);
      a.zc[orow] = zv;
    }
  } else {
    if ((lane & (32 / RPW - 1)) == 0) st_relaxed(a.dout + orow, double(tot));
  }
}

template <class T, class A, bool FWD>
__global__ void __launch_bounds__(NTHR) k_trsv(TrsvArgs a) {
  using PL = Plan<(int)sizeof(T)>;
  extern __shared__ __align__(128) unsigned char dsm_trsv[];
  RowSmem sm;
  sm.ring = dsm_trsv;
  sm.zbuf = reinterpret_cast<double*>(dsm_trsv + PL::RING);
  sm.full = reinterpret_cast<unsigned long long*>(sm.zbuf + MAXST * TILE);
  sm.empty = sm.full + MAXST;
  sm.zbar = sm.empty + MAXST;
  __shared__ unsigned long long s_ticket;
  if (threadIdx.x == 0) {
    s_ticket = atomicAdd(a.ticket, 1ull);
    for (int k = 0; k < MAXST; ++k) {
      mbar_init(&sm.full[k], 1);
      mbar_init(&sm.empty[k], NCONS / 32);
      mbar_init(&sm.zbar[k], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int t = (int)(s_ticket % (unsigned long long)a.nwork);
  const TrsvWork wk = a.work[t];
  const MatDesc md = a.md[wk.mat];
  if (a.sc && a.sc[md.sub].done) return;
  if (md.coarse) {
    // a full-row FP64 coarse item needs a 32 KB stage: FP64 launches only (host checks)
    bool done = false;
    if constexpr (sizeof(T) == 8) {
      if (md.nsub == 1) {
        sweep_item<double, double, 64, FWD, PL::RING>(a, a.ctiles, a.cut, wk.mat, wk.row, 0, md.cb, sm);
        done = true;
      }
    }
    if (!done) {
      if (md.nsub == 2)
        sweep_item<double, double, 32, FWD, PL::RING>(a, a.ctiles, a.cut, wk.mat, wk.row, wk.slab,
                                                       md.cb, sm);
      else
        sweep_item<double, double, 16, FWD, PL::RING>(a, a.ctiles, a.cut, wk.mat, wk.row, wk.slab,
                                                       md.cb, sm);
    }
  } else {
    const T* lt = reinterpret_cast<const T*>(a.ltiles);
    const T* ut = reinterpret_cast<const T*>(a.lut);
    if (md.nsub == 2)
      sweep_item<T, A, 32, FWD, PL::RING>(a, lt, ut, wk.mat, wk.row, wk.slab, md.cb, sm);
    else if (md.nsub == 4)
      sweep_item<T, A, 16, FWD, PL::RING>(a, lt, ut, wk.mat, wk.row, wk.slab, md.cb, sm);
    else
      sweep_item<T, A, 64, FWD, PL::RING>(a, lt, ut, wk.mat, wk.row, 0, md.cb, sm);
  }
}

__global__ void k_fill_pending(double* p, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    p[i] = __longlong_as_double((long long)TRSV_PENDING);
}

void launch_fill_pending(double* p, long long n, cudaStream_t s) {
  k_fill_pending<<<152 * 4, 256, 0, s>>>(p, n);
}

template <class T, class A, bool FWD>
static void launch_k(const TrsvArgs& a, cudaStream_t s, int grid = 0) {
  constexpr int bytes = Plan<(int)sizeof(T)>::BYTES;
  cudaFuncSetAttribute(k_trsv<T, A, FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  k_trsv<T, A, FWD><<<grid > 0 ? grid : a.nwork, NTHR, bytes, s>>>(a);
}

void launch_trsv_fwd(const TrsvArgs& a, Store st, cudaStream_t s, int grid) {
  switch (st) {
    case Store::F64: launch_k<double, double, true>(a, s, grid); break;
    case Store::F32: launch_k<float, float, true>(a, s, grid); break;
    default: launch_k<__nv_bfloat16, float, true>(a, s, grid); break;
  }
}

void launch_trsv_bwd(const TrsvArgs& a, Store st, cudaStream_t s) {
  switch (st) {
    case Store::F64: launch_k<double, double, false>(a, s); break;
    case Store::F32: launch_k<float, float, false>(a, s); break;
    default: launch_k<__nv_bfloat16, float, false>(a, s); break;
  }
}

}  // namespace sfcdd
