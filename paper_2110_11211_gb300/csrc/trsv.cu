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
// Zero rows: rows nzr[I].. of tile row I are zero in all its off-block Lh
// tiles (the factor keeps the narrow local bands), so the forward neither
// streams nor applies them, and the backward reads only the left halves of
// transposed tiles whose source bound is at most 32.
//
// Parallel layout: one CTA per work item.  A local matrix is either one item
// (the whole matrix, its tile rows chained through shared memory: see
// sweep_matrix) or one item per (tile row, slab); coarse rows are always slab
// items, in the same launch.  A slab is R = 64 / S consecutive rows of the tile
// row (S = 1, 2 or 4 per matrix: splitting the rows of a long chain spreads its
// FP64 GEMVs over S SMs).  CTAs
// take tickets from a monotone counter and map them through a work list in
// which every item comes after the items it depends on, so a CTA only ever
// waits for CTAs that already started (no deadlock, whatever the residency).
// Row results are their own ready flags: before a launch the result slots hold
// a sentinel NaN bit pattern, every slot is written exactly once per launch
// with a relaxed store, and a consumer polls the slots it needs with relaxed
// loads until none holds the sentinel (bounded spin; a timeout sets the error
// word and the CTA still drains its copies before it returns).  One polling
// warp, which does no arithmetic, waits for the 64 values of each dependency
// and hands them to the eight consumer warps through shared memory and a
// per-stage mbarrier: one straggling lane cannot hold up eight warps, the L2
// sees one poller per CTA, and the poller runs ahead of the consumers, so its
// round trips to L2 overlap their GEMVs on the previous tiles.  The forward
// launch resets the backward slots of its slab and also writes its results to
// a plain buffer zc; the backward launch reads z from zc and resets the forward
// slots of its slab (nothing reads them during the backward launch).
//
// Data movement: a producer warp streams the item's tile slabs (E tiles first
// in the backward) from HBM into a shared-memory ring with bulk asynchronous
// copies (cp.async.bulk, completion on mbarriers); eight consumer warps wait on
// the ring's mbarriers, apply the slabs, and free the stages.  In launches of
// slab items only, the ring holds 64 KB for a single problem (two FP64 tiles,
// four FP32, eight BF16; three CTAs per SM) and 32 KB for a batch (more CTAs
// per SM); coarse items of low-precision launches run in 16- or 32-row slabs.
// Launches with whole-matrix items use eight 32-row pieces (FP64 128 KB) and
// the matrix vector instead (see Plan).
#include "sfcdd_internal.cuh"

namespace sfcdd {

constexpr int NCONS = 256;                 // consumer threads: 8 warps
constexpr int PROD0 = NCONS + 32;          // + one polling warp, then the producer warp
constexpr int NTHR = PROD0 + 32;
constexpr int MAXST = 8;
constexpr long long SPIN_LIMIT = 1ll << 22;
constexpr long long MBAR_LIMIT = 1ll << 26;
constexpr long long SPIN_FAST = 1 << 12;   // polls before the poller starts to back off

// Shared-memory plan of a launch whose local factors have element size ES.
template <int ES, bool WHOLE = false, bool BIG = false>
struct Plan {
  // Slab launches, BIG (TrsvArgs::wide_ring): 64 KB (two FP64 tiles, four FP32,
  // eight BF16), three CTAs per SM; against 32 KB it gives the coarse slab items
  // of a single large problem more stages in flight (FP32 local factors: 360 ->
  // 339 us per PCG iteration); 128 KB leaves too few CTAs.  Otherwise 32 KB
  // (one FP64 tile, two FP32, four BF16 in 16 KB): more CTAs per SM, which the
  // many small matrices of a batch need (the 385-subgrid batch: FP32 solve 60
  // ms against 80 with 64 KB).  Launches with whole-matrix items: eight 32-row
  // pieces (FP64 128 KB: a CTA streams the whole matrix and needs the bytes in
  // flight of an SM), plus the matrix vector.  BIG: FP32 and BF16 launches take
  // the FP64 ring size too when the matrix vector still fits, so that one CTA
  // holds an SM and the coarse row items of the launch get eight 32-row stages:
  // two whole-matrix sweeps on one SM, or a sweep beside coarse items with four
  // stages, were measured slower (FP32 local factors: 418 -> 308 us per PCG
  // iteration).
  static constexpr int RING = WHOLE ? 8 * 32 * TILE * (BIG ? 8 : ES)
                                    : (BIG ? 64 * 1024 : (ES == 8 ? 1 : 2) * TILE2 * ES);
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
// Factor tiles are read once per substitution and stream through L2: their
// bulk copies carry an evict-first policy, so that they do not push the PCG
// vectors, the result slots and the index maps (tens of MB, reused every
// iteration) out of L2.
__device__ __forceinline__ unsigned long long evict_first_policy() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void factor_copy(void* dst, const void* src, unsigned bytes,
                                            unsigned long long* bar, unsigned long long pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
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

// One element of a shared-memory slab row as the accumulation type.
__device__ __forceinline__ double sm_one(const double* p) { return *p; }
__device__ __forceinline__ float sm_one(const float* p) { return *p; }
__device__ __forceinline__ float sm_one(const __nv_bfloat16* p) {
  return __uint_as_float((unsigned)*reinterpret_cast<const unsigned short*>(p) << 16);
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
  // Zero rows of the off-block tiles.  Forward: only the slab's rows below the
  // tile row's bound are streamed and applied (none: z = b).  Backward: an Lh^T
  // tile whose source row bound is at most TILE / 2 has its nonzeros in the left
  // half of every row; only those halves are streamed and applied, against the
  // first TILE / 2 entries of x_c.
  int nrow = R;
  if (FWD && a.ts.nzr) {
    nrow = min(R, max(0, a.ts.nzr[fb + r] - R * slab));
    if (nrow == 0) ntile = 0;
  }
  auto half_tile = [&](int t) {
    return !FWD && t >= nE && a.ts.nzr != nullptr && a.ts.nzr[fb + cl[ncl - 1 - (t - nE)]] <= TILE / 2;
  };
  // dependency vector of tile tt: z of the block comes from the forward launch
  // (a previous kernel, never the sentinel), the other vectors from this launch
  auto dep = [&](int tt) -> const double* {
    return FWD       ? a.y + vb + (k0 + tt) * TILE
           : tt < nE ? a.zc + vb + (blk0 + tt) * TILE
                     : a.dout + vb + cl[ncl - 1 - (tt - nE)] * TILE;
  };
  if (threadIdx.x >= PROD0) {
    // producer warp: every lane waits for the stage; lane 0 issues the copy
    const int pl = threadIdx.x - PROD0;
    const unsigned long long pol = evict_first_policy();
    for (int t = 0; t < ntile; ++t) {
      const int s = t % NS, k = t / NS;
      if (k >= 1) mbar_wait(&sm.empty[s], (k - 1) & 1, a.err, 10);
      unsigned char* dst = sm.ring + (size_t)s * SB;
      const T* src;
      unsigned bytes = SB;
      if (FWD) {
        src = row0 + (long long)t * TILE2;
        bytes = (unsigned)(nrow * TILE * (int)sizeof(T));
      } else if (t < nE) {
        // E(r, kp): ut holds the block's lower tiles, the tiles array its upper ones
        const int kp = blk0 + t;
        src = (kp <= r ? ut + tile_at(a.ts, tb, fb, r, kp) : lt + tile_at(a.ts, tb, fb, kp, r)) +
              soff;
      } else {
        src = ut + tile_at(a.ts, tb, fb, cl[ncl - 1 - (t - nE)], r) + soff;
      }
      // half tiles: FP64 slots hold the left halves packed (launch_pack_half_tiles),
      // so the slab's R half rows are one contiguous copy; narrower types keep
      // the full slab (their rows' halves are too short to pay)
      if (sizeof(T) == 8 && half_tile(t)) {
        constexpr unsigned HB = TILE / 2 * sizeof(T);
        src = ut + tile_at(a.ts, tb, fb, cl[ncl - 1 - (t - nE)], r) +
              (long long)R * slab * (TILE / 2);
        bytes = R * HB;
      }
      if (pl == 0) {
        mbar_expect_tx(&sm.full[s], bytes);
        factor_copy(dst, src, bytes, &sm.full[s], pol);
      }
    }
    return;
  }
  if (threadIdx.x >= NCONS) {
    // polling warp: waits for each tile's dependency values and hands them to
    // the consumers through shared memory, running ahead of them by up to NS
    // tiles, so that its round trips to L2 overlap their GEMVs
    const int pln = threadIdx.x & 31;
    for (int t = 0; t < ntile; ++t) {
      const int s = t % NS;
      double* zs = sm.zbuf + s * TILE;
      // the consumers are done with the previous use of zs (stage s)
      if (t >= NS) mbar_wait(&sm.empty[s], ((t / NS) & 1) ^ 1, a.err, 13);
      if (!half_tile(t) || pln < TILE / 4) {
        const double2 v = wait_pair(dep(t) + 2 * pln, a.err, FWD ? 1 : 2);
        *reinterpret_cast<double2*>(zs + 2 * pln) = v;
      }
      __syncwarp();
      if (pln == 0) mbar_arrive(&sm.zbar[s]);
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
    const bool half = half_tile(t);
    double2 v = make_double2(0.0, 0.0);
    mbar_wait(&sm.zbar[s], ph, a.err, 14);
    if (!half) v = *reinterpret_cast<const double2*>(zs + 2 * lane);
    mbar_wait(&sm.full[s], ph, a.err, 11);
    const T* st = reinterpret_cast<const T*>(sm.ring + (size_t)s * SB);
    if (half) {
      // - Lh^T x on the left half: column `lane`
      const A vh = A(-zs[lane]);
      constexpr int HS = sizeof(T) == 8 ? TILE / 2 : TILE;  // row stride of a half tile's stage
#pragma unroll
      for (int i = 0; i < RPW; ++i) acc[i] = fma(sm_one(st + (rloc + i) * HS + lane), vh, acc[i]);
    } else {
      // backward: + E z, - Lh^T x
      const bool neg = !FWD && t >= nE;
      const A v0 = A(neg ? -v.x : v.x), v1 = A(neg ? -v.y : v.y);
#pragma unroll
      for (int i = 0; i < RPW; ++i) {
        if (FWD && rloc + i >= nrow) break;  // zero rows (not streamed)
        A l0, l1;
        sm_pair(st + (rloc + i) * TILE + 2 * lane, l0, l1);
        acc[i] = fma(l0, v0, acc[i]);
        acc[i] = fma(l1, v1, acc[i]);
      }
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

// ---------------------------------------------------------------------------
// Whole-matrix items: one CTA sweeps every tile row of a local matrix (cb = 1,
// zero-row bounds known), so the row-to-row chain passes through shared
// memory and a CTA barrier instead of result slots in L2 polled by other CTAs.
// With the narrow bands of curve-ordered subdomains the chain carries about one
// off-block tile per row, which makes the cross-CTA hand-off the bound of the
// row-slab items; here a forward step costs the tile's FMAs and one barrier,
// and a backward step only the product with the previous row's x and an
// mbarrier phase (the rest of the row's work is formed before the wait).  The
// matrix vector (z, then x) lives in shared memory.
//   forward   z_I = b_I - sum_{K < I} Lh_IK z_K   (rows below nzr[I]: z = b)
//   backward  x_I = E_I z_I - sum_{K > I} Lh_KI^T x_K  (columns below nzr[K])
// The producer warp streams the factor in pieces of 32 tile rows (forward: the
// nonzero rows of each off-block tile; backward: the two halves of E_I, then
// per Lh^T tile its left halves (FP64, nzr[K] <= TILE / 2: 64 rows of 32
// columns, packed) or its two halves, the nearest row's tile last) through an
// eight-stage ring.  Consumer
// thread (j, g) = (tid / 8, tid % 8) owns tile rows j and j + 32 and the
// 16-byte chunks g + 8 k of a piece row, so each quarter-warp phase of a
// shared load reads one contiguous 128-byte row segment.
__device__ __forceinline__ void consumers_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// Right-hand side of local row grow of matrix m (zero beyond its size).
__device__ __forceinline__ double local_rhs(const TrsvArgs& a, const MatDesc& md, int vb, int n,
                                            int grow) {
  if (grow >= n) return 0.0;
  int pos;
  if (a.ts.lperm) {
    pos = a.ts.lperm[vb + grow];
  } else {
    pos = md.start + grow;
    if (pos >= md.rhs_len) pos -= md.rhs_len;
  }
  return a.rhs[md.rhs_base + pos];
}

// acc += sum over the thread's CH chunks of one piece row (EPC elements each)
// times the matching entries of the vector slice xs.
template <class T, class A, int CH>
__device__ __forceinline__ void piece_row_dot(const T* __restrict__ row, int g, const A* xs, A& acc) {
  constexpr int EPC = 16 / (int)sizeof(T);
#pragma unroll
  for (int k = 0; k < CH; ++k) {
    const T* p = row + (g + 8 * k) * EPC;
#pragma unroll
    for (int e = 0; e < EPC; e += 2) {
      A l0, l1;
      sm_pair(p + e, l0, l1);
      acc = fma(l0, xs[k * EPC + e], acc);
      acc = fma(l1, xs[k * EPC + e + 1], acc);
    }
  }
}

template <class A>
__device__ __forceinline__ A sum8(A v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  return v;
}

// Both sums of (a0, a1) over the 8-lane group at once: the first exchange halves
// the work (lanes with bit 2 clear keep a0, the others a1), three adds instead
// of six.  Returns a0's total in lanes g < 4 and a1's in lanes g >= 4.
template <class A>
__device__ __forceinline__ A sum8_pair(A a0, A a1) {
  const bool hi = (threadIdx.x & 4) != 0;
  A v = (hi ? a1 : a0) + __shfl_xor_sync(0xffffffffu, hi ? a0 : a1, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

template <class T, class A, bool FWD, int RING>
__device__ void sweep_matrix(const TrsvArgs& a, const T* __restrict__ lt, const T* __restrict__ ut,
                             int m, const RowSmem& sm, double* __restrict__ zv) {
  constexpr int PR = 32;                                   // rows of a piece
  constexpr unsigned PB = PR * TILE * sizeof(T);           // piece bytes
  constexpr int NS = (RING / (int)PB) < MAXST ? (RING / (int)PB) : MAXST;
  constexpr int EPC = 16 / (int)sizeof(T);                 // elements per 16-byte chunk
  constexpr int CH = TILE / EPC / 8;                       // chunks of a full row per thread
  constexpr unsigned HB = TILE / 2 * sizeof(T);            // half a tile row
  static_assert(NS >= 2, "whole-matrix ring needs two pieces");
  const long long tb = a.ts.tbase[m];
  const int vb = a.ts.vbase[m];
  const int fb = vb / TILE;
  const int nt = a.ts.nt[m];
  auto half_piece = [&](int K) { return sizeof(T) == 8 && a.ts.nzr[fb + K] <= TILE / 2; };

  if (threadIdx.x >= NCONS && threadIdx.x < PROD0) return;  // no polling: the chain is in the CTA
  if (threadIdx.x >= PROD0) {
    // producer warp: the pieces in consumption order
    const int pl = threadIdx.x - PROD0;
    const unsigned long long pol = evict_first_policy();
    int t = 0;
    auto put = [&](const T* src, unsigned bytes) {
      const int s = t % NS, k = t / NS;
      if (k >= 1) mbar_wait(&sm.empty[s], (k - 1) & 1, a.err, 20);
      unsigned char* dst = sm.ring + (size_t)s * PB;
      if (pl == 0) {
        mbar_expect_tx(&sm.full[s], bytes);
        factor_copy(dst, src, bytes, &sm.full[s], pol);
      }
      ++t;
    };
    if (FWD) {
      for (int I = 0; I < nt; ++I) {
        const int nz = a.ts.nzr[fb + I];
        for (int K = a.ts.kmin[fb + I]; K < I; ++K)
          for (int p = 0; p * PR < nz; ++p)
            put(lt + tile_at(a.ts, tb, fb, I, K) + (long long)p * PR * TILE,
                (unsigned)(min(PR, nz - p * PR) * TILE * (int)sizeof(T)));
      }
    } else {
      if (pl == 0) {
        const unsigned zb = (unsigned)(nt * TILE * (int)sizeof(double));
        mbar_expect_tx(&sm.zbar[0], zb);
        bulk_copy(zv, a.zc + vb, zb, &sm.zbar[0]);
      }
      for (int I = nt - 1; I >= 0; --I) {
        const T* e = ut + tile_at(a.ts, tb, fb, I, I);
        put(e, PB);
        put(e + PR * TILE, PB);
        const int* cl = a.ts.colidx + a.ts.colptr[fb + I];
        const int ncl = a.ts.colptr[fb + I + 1] - a.ts.colptr[fb + I];
        for (int q = 1; q <= ncl; ++q) {
          const int K = cl[q < ncl ? q : 0];  // the nearest row last (it waits for the chain)
          const T* src = ut + tile_at(a.ts, tb, fb, K, I);
          if (half_piece(K)) {
            put(src, TILE * HB);  // the left halves, packed in the slot (launch_pack_half_tiles)
          } else {
            put(src, PB);
            put(src + PR * TILE, PB);
          }
        }
      }
    }
    return;
  }

  const int tid = threadIdx.x, lane = tid & 31;
  const int j = tid >> 3, g = tid & 7;
  const MatDesc md = a.md[m];
  const int n = a.ts.n[m];
  int t = 0;
  // next piece: wait for it; returns its rows
  auto take = [&]() -> const T* {
    const int s = t % NS;
    mbar_wait(&sm.full[s], (t / NS) & 1, a.err, 21);
    return reinterpret_cast<const T*>(sm.ring + (size_t)s * PB);
  };
  auto give = [&]() {
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.empty[t % NS]);
    ++t;
  };
  // the thread's entries of a full vector tile: chunks g + 8 k
  auto slice = [&](int K, A (&xs)[CH * EPC], bool neg) {
#pragma unroll
    for (int k = 0; k < CH; ++k)
#pragma unroll
      for (int e = 0; e < EPC; ++e) {
        const double v = zv[K * TILE + (g + 8 * k) * EPC + e];
        xs[k * EPC + e] = A(neg ? -v : v);
      }
  };

  if (FWD) {
    // the right-hand side, gathered once: zv holds b_I until z_I replaces it
    for (int r = tid; r < nt * TILE; r += NCONS) zv[r] = local_rhs(a, md, vb, n, r);
    consumers_sync();
    for (int I = 0; I < nt; ++I) {
      const int r0 = I * TILE + j, r1 = r0 + PR;
      const int nz = a.ts.nzr[fb + I];
      A acc0 = A(0), acc1 = A(0);
      for (int K = a.ts.kmin[fb + I]; K < I; ++K) {
        A xs[CH * EPC];
        slice(K, xs, false);
        for (int p = 0; p * PR < nz; ++p) {
          const T* st = take();
          if (j < nz - p * PR) piece_row_dot<T, A, CH>(st + j * TILE, g, xs, p ? acc1 : acc0);
          give();
        }
      }
      if (nz > PR) {  // rows of both pieces: lane 0 gets acc0's total, lane 4 acc1's
        const A tot = sum8_pair(acc0, acc1);
        acc0 = __shfl_sync(0xffffffffu, tot, lane & ~7);
        acc1 = __shfl_sync(0xffffffffu, tot, (lane & ~7) | 4);
      } else {        // uniform over the CTA: the second piece is empty
        acc0 = sum8(acc0);
      }
      if (g == 0) {
        const double z0 = double(A(zv[r0]) - acc0), z1 = double(A(zv[r1]) - acc1);
        zv[r0] = z0;
        zv[r1] = z1;
        a.y[vb + r0] = z0;
        a.y[vb + r1] = z1;
        a.zc[vb + r0] = z0;
        a.zc[vb + r1] = z1;
        // the backward slots, polled by row-slab items of other launches
        a.dout[vb + r0] = __longlong_as_double((long long)TRSV_PENDING);
        a.dout[vb + r1] = __longlong_as_double((long long)TRSV_PENDING);
      }
      consumers_sync();  // z_I visible to the next rows
    }
  } else {
    // E_I z_I and the products with the x_K of rows K >= I + 2 do not wait for
    // the chain: every warp forms them first and waits only before the product
    // with x_{I+1}, on an mbarrier (zbar[1], NCONS / 32 arrivals, set up by
    // k_trsv) at which each warp arrives once it has written its rows of
    // x_{I+1}.  A warp reads z_I into registers before it arrives for x_{I+1};
    // x_I replaces z_I in zv only after every warp has arrived, so those reads
    // never race with the writes.
    unsigned long long* xbar = &sm.zbar[1];
    mbar_wait(&sm.zbar[0], 0, a.err, 22);  // z in zv
    auto apply_lt = [&](int K, A& acc0, A& acc1) {
      if (half_piece(K)) {
        // 64 rows of 32 columns: chunks g and g + 8 of rows j and j + 32
        A xs[2 * EPC];
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
          for (int e = 0; e < EPC; ++e) xs[k * EPC + e] = A(-zv[K * TILE + (g + 8 * k) * EPC + e]);
        const T* st = take();
        piece_row_dot<T, A, 2>(st + j * (TILE / 2), g, xs, acc0);
        piece_row_dot<T, A, 2>(st + (j + PR) * (TILE / 2), g, xs, acc1);
        give();
      } else {
        A xs[CH * EPC];
        slice(K, xs, true);
        const T* st = take();
        piece_row_dot<T, A, CH>(st + j * TILE, g, xs, acc0);
        give();
        st = take();
        piece_row_dot<T, A, CH>(st + j * TILE, g, xs, acc1);
        give();
      }
    };
    A zs[CH * EPC];
    slice(nt - 1, zs, false);
    consumers_sync();  // every warp holds z_{nt-1} before x_{nt-1} replaces it
    for (int I = nt - 1; I >= 0; --I) {
      A acc0 = A(0), acc1 = A(0);
      const T* st = take();
      piece_row_dot<T, A, CH>(st + j * TILE, g, zs, acc0);
      give();
      st = take();
      piece_row_dot<T, A, CH>(st + j * TILE, g, zs, acc1);
      give();
      const int* cl = a.ts.colidx + a.ts.colptr[fb + I];
      const int ncl = a.ts.colptr[fb + I + 1] - a.ts.colptr[fb + I];
      for (int q = 1; q < ncl; ++q) apply_lt(cl[q], acc0, acc1);  // rows >= I + 2
      if (I < nt - 1) mbar_wait(xbar, (unsigned)(nt - 2 - I) & 1u, a.err, 23);  // x_{I+1}
      if (ncl > 0) apply_lt(cl[0], acc0, acc1);
      // lane g = 0 of the group writes row j (acc0's total), lane g = 4 row j + 32
      const A tot = sum8_pair(acc0, acc1);
      if (I > 0) slice(I - 1, zs, false);
      if ((g & 3) == 0) {
        const int row = I * TILE + j + (g ? PR : 0);
        zv[row] = double(tot);
        a.dout[vb + row] = double(tot);
        // the forward slot, polled by row-slab items of other launches
        a.y[vb + row] = __longlong_as_double((long long)TRSV_PENDING);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(xbar);  // this warp's rows of x_I are in zv
    }
  }
}

template <class T, class A, bool FWD, bool WHOLE, bool BIG = false>
__global__ void __launch_bounds__(NTHR) k_trsv(TrsvArgs a) {
  using PL = Plan<(int)sizeof(T), WHOLE, BIG>;
  extern __shared__ __align__(128) unsigned char dsm_trsv[];
  RowSmem sm;
  sm.ring = dsm_trsv;
  sm.zbuf = reinterpret_cast<double*>(dsm_trsv + PL::RING);
  sm.full = reinterpret_cast<unsigned long long*>(sm.zbuf + MAXST * TILE);
  sm.empty = sm.full + MAXST;
  sm.zbar = sm.empty + MAXST;
  __shared__ unsigned long long s_ticket;
  if (threadIdx.x == 0) {
    const unsigned long long tk = atomicAdd(a.ticket, 1ull);
    s_ticket = tk;
    // the backward sweep of a whole-matrix item takes zbar[1] as the phase
    // barrier of its rows of x, one arrival per consumer warp
    const bool whole_item = WHOLE && a.work[(int)(tk % (unsigned long long)a.nwork)].row < 0;
    for (int k = 0; k < MAXST; ++k) {
      mbar_init(&sm.full[k], 1);
      mbar_init(&sm.empty[k], NCONS / 32);
      mbar_init(&sm.zbar[k], whole_item && k == 1 ? NCONS / 32 : 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int t = (int)(s_ticket % (unsigned long long)a.nwork);
  const TrsvWork wk = a.work[t];
  const MatDesc md = a.md[wk.mat];
  if (a.sc && a.sc[md.sub].done) return;
  if (wk.row < 0) {
    if constexpr (WHOLE)
      sweep_matrix<T, A, FWD, PL::RING>(a, reinterpret_cast<const T*>(a.ltiles),
                                        reinterpret_cast<const T*>(a.lut), wk.mat, sm,
                                        reinterpret_cast<double*>(dsm_trsv + PL::BYTES));
    return;
  }
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

// Shared memory of a launch with whole-matrix items (largest local tile count
// max_nt), and whether it fits a CTA.
constexpr long long CTA_SMEM_MAX = 227 * 1024;
template <int ES>
static long long whole_bytes(int max_nt) {
  return Plan<ES, true>::BYTES + (long long)max_nt * TILE * (long long)sizeof(double);
}

bool whole_fits(Store st, int max_nt) {
  if (max_nt <= 0) return false;
  const long long b = st == Store::F64 ? whole_bytes<8>(max_nt)
                      : st == Store::F32 ? whole_bytes<4>(max_nt)
                                         : whole_bytes<2>(max_nt);
  return b <= CTA_SMEM_MAX;
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
  const int nblk = grid > 0 ? grid : a.nwork;
  if (a.zv_doubles > 0) {
    const long long zb = (long long)a.zv_doubles * (long long)sizeof(double);
    if (sizeof(T) < 8 && Plan<(int)sizeof(T), true, true>::BYTES + zb <= CTA_SMEM_MAX) {
      const int bytes = (int)(Plan<(int)sizeof(T), true, true>::BYTES + zb);
      cudaFuncSetAttribute(k_trsv<T, A, FWD, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           bytes);
      k_trsv<T, A, FWD, true, true><<<nblk, NTHR, bytes, s>>>(a);
      return;
    }
    const int bytes = (int)(Plan<(int)sizeof(T), true>::BYTES + zb);
    cudaFuncSetAttribute(k_trsv<T, A, FWD, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    k_trsv<T, A, FWD, true><<<nblk, NTHR, bytes, s>>>(a);
  } else if (a.wide_ring) {
    constexpr int bytes = Plan<(int)sizeof(T), false, true>::BYTES;
    cudaFuncSetAttribute(k_trsv<T, A, FWD, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         bytes);
    k_trsv<T, A, FWD, false, true><<<nblk, NTHR, bytes, s>>>(a);
  } else {
    constexpr int bytes = Plan<(int)sizeof(T)>::BYTES;
    cudaFuncSetAttribute(k_trsv<T, A, FWD, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    k_trsv<T, A, FWD, false><<<nblk, NTHR, bytes, s>>>(a);
  }
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
