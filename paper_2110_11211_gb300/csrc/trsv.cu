// Batched forward / backward substitution with the Cholesky factors of the
// local matrices A_i and of the coarse matrix A_0 (Algorithm 2, steps 2-3: the
// factorization is done once in the setup phase and every application of the
// preconditioner only runs the two triangular solves, Sec. 3.1).
//
// Parallel layout: one CTA per (matrix, tile row).  CTAs take tickets from a
// monotone counter and map them through a work list in which every tile row
// comes after the rows it depends on, so a CTA only ever waits for CTAs that
// already started (no deadlock, whatever the residency).
// Row results are their own ready flags: before a launch the result slots hold
// a sentinel NaN bit pattern (the forward launch resets the backward slots of
// its rows, the backward launch resets the forward slots of its rows after
// reading them; setup fills both), every slot is written exactly once per
// launch with a relaxed store, and a consumer polls the slots it needs with
// relaxed loads until none holds the sentinel (bounded spin; a timeout sets the
// error word and the CTA still drains its copies before it returns).
// The diagonal slot of every tile row holds the inverse of the diagonal block,
// so both the off-diagonal updates and the diagonal solve are GEMVs.
//
// Data movement: a producer warp streams the row's tiles from HBM into a
// shared-memory ring with bulk asynchronous copies (cp.async.bulk, completion
// on mbarriers), the diagonal tile first into its own buffer; eight consumer
// warps wait on the ring's mbarriers, apply the tiles, and free the slots.
// Everything a row needs that does not depend on other rows (its right-hand
// side, the diagonal tile, its tile list) is fetched before the first wait, so
// the dependency chain between rows only carries the flag, one tile and the
// diagonal GEMV.
#include "sfcdd_internal.cuh"

namespace sfcdd {

constexpr int NCONS = 256;                 // consumer threads: 8 warps x 8 rows
constexpr int NTHR = NCONS + 32;           // + one producer warp
constexpr int RING_BYTES = 64 * 1024;      // tile ring (2 FP64 / 4 FP32 / 8 BF16 tiles)
constexpr int DIAG_BYTES = TILE2 * 8;      // diagonal tile buffer (room for FP64)
constexpr int MAXST = 8;
constexpr long long SPIN_LIMIT = 1ll << 22;
constexpr long long MBAR_LIMIT = 1ll << 26;

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
__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(NCONS) : "memory");
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
    if (++it > 32) __nanosleep(20);
    if ((it & 1023) == 0 &&
        (*((volatile int*)&err->code) != 0 || it > SPIN_LIMIT)) {
      if (atomicCAS(&err->code, 0, (int)SFCDD_ERR_TIMEOUT) == 0) err->index = site;
      break;
    }
    v = ld_relaxed2(p);
  }
  return v;
}

// Two consecutive elements of a shared-memory tile row as the accumulation type.
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

// Sum over the 32 lanes of v[i] for the warp's 8 rows in 9 shuffles (halving
// exchanges then a 4-lane reduction).  Every lane returns the total of row
// `row` = (lane >> 2) & 7.
template <class A>
__device__ __forceinline__ A reduce8(A (&v)[8], int& row) {
  const int lane = threadIdx.x & 31;
  A w4[4], w2[2];
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const A keep = h16 ? v[i + 4] : v[i];
    const A send = h16 ? v[i] : v[i + 4];
    w4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const A keep = h8 ? w4[i + 2] : w4[i];
    const A send = h8 ? w4[i] : w4[i + 2];
    w2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const A keep = h4 ? w2[1] : w2[0];
  const A send = h4 ? w2[0] : w2[1];
  A t = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  t += __shfl_xor_sync(0xffffffffu, t, 2);
  t += __shfl_xor_sync(0xffffffffu, t, 1);
  row = (h16 ? 4 : 0) + (h8 ? 2 : 0) + (h4 ? 1 : 0);
  return t;
}

struct RowSmem {
  unsigned char* ring;
  unsigned char* diag;
  unsigned long long* full;   // [MAXST]
  unsigned long long* empty;  // [MAXST]
  unsigned long long* dbar;
  double* xs;                 // [TILE]
  double* red;                // [8 * TILE]
};

template <class T>
struct Ring {
  static constexpr unsigned TB = TILE2 * sizeof(T);
  static constexpr int NS = (RING_BYTES / (int)TB) < MAXST ? (RING_BYTES / (int)TB) : MAXST;
};

// Producer: the diagonal tile, then the row's tiles in consumption order.
template <class T, class TileAt>
__device__ void produce(const RowSmem& sm, int ntile, TileAt tile_k, const T* diag_tile,
                        ErrWord* err) {
  constexpr unsigned TB = Ring<T>::TB;
  constexpr int NS = Ring<T>::NS;
  mbar_expect_tx(sm.dbar, TB);
  bulk_copy(sm.diag, diag_tile, TB, sm.dbar);
  for (int t = 0; t < ntile; ++t) {
    const int s = t % NS, k = t / NS;
    if (k >= 1) mbar_wait(&sm.empty[s], (k - 1) & 1, err, 10);
    mbar_expect_tx(&sm.full[s], TB);
    bulk_copy(sm.ring + (size_t)s * TB, tile_k(t), TB, &sm.full[s]);
  }
}

// Forward row r of matrix m: y_r = Linv_rr (g_r - sum_{c<r} L_rc y_c).
template <class T, class A>
__device__ void fwd_row(const TrsvArgs& a, const T* __restrict__ tiles, int m, int r,
                        const RowSmem& sm) {
  constexpr unsigned TB = Ring<T>::TB;
  constexpr int NS = Ring<T>::NS;
  const long long tb = a.ts.tbase[m];
  const int n = a.ts.n[m];
  const int vb = a.ts.vbase[m];
  const int fb = vb / TILE;
  const int k0 = a.ts.kmin[fb + r];
  const T* row0 = tiles + tb + (long long)a.ts.rowoff[fb + r] * TILE2;  // tile (r, k0)
  const int ntile = r - k0;
  if (threadIdx.x >= NCONS) {
    if (threadIdx.x == NCONS)
      produce<T>(sm, ntile, [=](int t) { return row0 + (long long)t * TILE2; },
                 row0 + (long long)ntile * TILE2, a.err);
    return;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // right-hand side of this warp's rows (independent of other rows)
  double gval = 0.0;
  if (lane < 8) {
    const int grow = r * TILE + 8 * w + lane;
    if (grow < n) {
      const MatDesc md = a.md[m];
      if (md.coarse) {
        gval = a.g0[md.rhs_base + grow];
      } else {
        int pos;
        if (a.ts.lperm) {
          pos = a.ts.lperm[vb + grow];
        } else {
          pos = md.start + grow;
          if (pos >= md.rhs_len) pos -= md.rhs_len;
        }
        gval = a.rhs[md.rhs_base + pos];
      }
    }
  }
  // this row's backward slots are reset here (nobody reads them in this launch)
  if (threadIdx.x < TILE) a.dout[vb + r * TILE + threadIdx.x] = __longlong_as_double((long long)TRSV_PENDING);
  A part[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) part[i] = A(0);
  for (int t = 0; t < ntile; ++t) {
    const int s = t % NS;
    const double2 yv = wait_pair(a.y + vb + (k0 + t) * TILE + 2 * lane, a.err, 1);
    const A y0 = A(yv.x), y1 = A(yv.y);
    mbar_wait(&sm.full[s], (t / NS) & 1, a.err, 11);
    const T* st = reinterpret_cast<const T*>(sm.ring + (size_t)s * TB);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      A l0, l1;
      sm_pair(st + (8 * w + i) * TILE + 2 * lane, l0, l1);
      part[i] = fma(l0, y0, part[i]);
      part[i] = fma(l1, y1, part[i]);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.empty[s]);
  }
  int row;
  const A tot = reduce8(part, row);
  const double gr = __shfl_sync(0xffffffffu, gval, row);  // row r's rhs sits in lane r
  if ((lane & 3) == 0) sm.xs[8 * w + row] = double(A(gr) - tot);
  consumers_sync();
  // diagonal block: y_r = Linv_rr * xs
  mbar_wait(sm.dbar, 0, a.err, 12);
  const T* dt = reinterpret_cast<const T*>(sm.diag);
  const A x0 = A(sm.xs[2 * lane]), x1 = A(sm.xs[2 * lane + 1]);
  A q[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    A l0, l1;
    sm_pair(dt + (8 * w + i) * TILE + 2 * lane, l0, l1);
    q[i] = fma(l1, x1, l0 * x0);
  }
  const A yr = reduce8(q, row);
  if ((lane & 3) == 0) st_relaxed(a.y + vb + r * TILE + 8 * w + row, double(yr));
}

// Backward row r: d_r = Linv_rr^T (y_r - sum_{c>r} L_cr^T d_c).
template <class T, class A>
__device__ void bwd_row(const TrsvArgs& a, const T* __restrict__ tiles, int m, int r,
                        const RowSmem& sm) {
  constexpr unsigned TB = Ring<T>::TB;
  constexpr int NS = Ring<T>::NS;
  const long long tb = a.ts.tbase[m];
  const int vb = a.ts.vbase[m];
  const int fb = vb / TILE;
  // rows c > r whose envelope reaches column r (ascending), consumed from the last
  const int* cl = a.ts.colidx + a.ts.colptr[fb + r];
  const int ncl = a.ts.colptr[fb + r + 1] - a.ts.colptr[fb + r];
  if (threadIdx.x >= NCONS) {
    if (threadIdx.x == NCONS)
      produce<T>(sm, ncl,
                 [=](int t) { return tiles + tile_at(a.ts, tb, fb, cl[ncl - 1 - t], r); },
                 tiles + tile_at(a.ts, tb, fb, r, r), a.err);
    return;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // y_r comes from the forward launch (a previous kernel): plain loads are coherent;
  // the slot is then reset for the next forward launch (only this CTA reads it)
  double yown = 0.0;
  if (threadIdx.x < TILE) {
    yown = a.y[vb + r * TILE + threadIdx.x];
    a.y[vb + r * TILE + threadIdx.x] = __longlong_as_double((long long)TRSV_PENDING);
  }
  A p0 = A(0), p1 = A(0);
  for (int t = 0; t < ncl; ++t) {
    const int s = t % NS;
    const int c = cl[ncl - 1 - t];
    const double* dc = a.dout + vb + c * TILE + 8 * w;
    A dv[8];
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
      const double2 v = wait_pair(dc + i, a.err, 2);
      dv[i] = A(v.x);
      dv[i + 1] = A(v.y);
    }
    mbar_wait(&sm.full[s], (t / NS) & 1, a.err, 13);
    const T* st = reinterpret_cast<const T*>(sm.ring + (size_t)s * TB);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      A l0, l1;
      sm_pair(st + (8 * w + i) * TILE + 2 * lane, l0, l1);
      p0 = fma(l0, dv[i], p0);
      p1 = fma(l1, dv[i], p1);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.empty[s]);
  }
  sm.red[w * TILE + 2 * lane] = double(p0);
  sm.red[w * TILE + 2 * lane + 1] = double(p1);
  consumers_sync();
  if (threadIdx.x < TILE) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += sm.red[k * TILE + threadIdx.x];
    sm.xs[threadIdx.x] = double(A(yown) - A(s));
  }
  consumers_sync();
  mbar_wait(sm.dbar, 0, a.err, 14);
  const T* dt = reinterpret_cast<const T*>(sm.diag);
  A q0 = A(0), q1 = A(0);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    A l0, l1;
    sm_pair(dt + (8 * w + i) * TILE + 2 * lane, l0, l1);
    const A xv = A(sm.xs[8 * w + i]);
    q0 = fma(l0, xv, q0);
    q1 = fma(l1, xv, q1);
  }
  sm.red[w * TILE + 2 * lane] = double(q0);
  sm.red[w * TILE + 2 * lane + 1] = double(q1);
  consumers_sync();
  if (threadIdx.x < TILE) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += sm.red[k * TILE + threadIdx.x];
    st_relaxed(a.dout + vb + r * TILE + threadIdx.x, double(A(s)));
  }
}

constexpr int SMEM_BYTES =
    RING_BYTES + DIAG_BYTES + (2 * MAXST + 1) * 8 + TILE * 8 + 8 * TILE * 8 + 16;

template <class T, class A, bool FWD>
__global__ void __launch_bounds__(NTHR) k_trsv(TrsvArgs a) {
  extern __shared__ __align__(128) unsigned char dsm_trsv[];
  RowSmem sm;
  sm.ring = dsm_trsv;
  sm.diag = dsm_trsv + RING_BYTES;
  sm.full = reinterpret_cast<unsigned long long*>(sm.diag + DIAG_BYTES);
  sm.empty = sm.full + MAXST;
  sm.dbar = sm.empty + MAXST;
  sm.xs = reinterpret_cast<double*>(sm.dbar + 1);
  sm.red = sm.xs + TILE;
  __shared__ unsigned long long s_ticket;
  if (threadIdx.x == 0) {
    s_ticket = atomicAdd(a.ticket, 1ull);
    for (int k = 0; k < MAXST; ++k) {
      mbar_init(&sm.full[k], 1);
      mbar_init(&sm.empty[k], NCONS / 32);
    }
    mbar_init(sm.dbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int t = (int)(s_ticket % (unsigned long long)a.nwork);
  const TrsvWork wk = a.work[t];
  const MatDesc md = a.md[wk.mat];
  if (a.sc && a.sc[md.sub].done) return;
  if (FWD) {
    if (md.coarse)
      fwd_row<double, double>(a, a.ctiles, wk.mat, wk.row, sm);
    else
      fwd_row<T, A>(a, reinterpret_cast<const T*>(a.ltiles), wk.mat, wk.row, sm);
  } else {
    if (md.coarse)
      bwd_row<double, double>(a, a.ctiles, wk.mat, wk.row, sm);
    else
      bwd_row<T, A>(a, reinterpret_cast<const T*>(a.ltiles), wk.mat, wk.row, sm);
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
static void launch_k(const TrsvArgs& a, cudaStream_t s) {
  cudaFuncSetAttribute(k_trsv<T, A, FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  k_trsv<T, A, FWD><<<a.nwork, NTHR, SMEM_BYTES, s>>>(a);
}

void launch_trsv_fwd(const TrsvArgs& a, Store st, cudaStream_t s) {
  switch (st) {
    case Store::F64: launch_k<double, double, true>(a, s); break;
    case Store::F32: launch_k<float, float, true>(a, s); break;
    default: launch_k<__nv_bfloat16, float, true>(a, s); break;
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
