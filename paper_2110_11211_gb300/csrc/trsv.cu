// Batched forward / backward substitution with the packed Cholesky factors of
// the local matrices A_i and of the coarse matrix A_0 (Algorithm 2, steps 2-3:
// the factorization is done once in the setup phase and every application of
// the preconditioner only runs the two triangular solves, Sec. 3.1).
//
// Parallel layout: one CTA per (matrix, tile row).  CTAs take tickets from a
// monotone counter and map them through a work list in which every tile row
// comes after the rows it depends on, so a CTA only ever waits for CTAs that
// already started (no deadlock, whatever the residency).  A finished row is
// published with a release store of the launch's epoch; consumers poll with
// acquire loads and a bounded spin (timeouts set the error word and return).
// The diagonal slot of every tile row holds the inverse of the diagonal block,
// so both the off-diagonal updates and the diagonal solve are GEMVs streaming
// tiles from HBM.
#include "sfcdd_internal.cuh"

namespace sfcdd {

constexpr int TB = 256;                   // threads per CTA: 8 warps x 8 rows
constexpr long long SPIN_LIMIT = 1ll << 22;

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Waits until *flag == epoch.  Returns false (after recording TIMEOUT) if the
// bounded spin ran out or another CTA already recorded an error.
__device__ __noinline__ bool wait_flag(const int* flag, int epoch, ErrWord* err, int site) {
  const int lane = threadIdx.x & 31;
  int ok = 1;
  if (lane == 0) {
    long long it = 0;
    while (ld_acquire(flag) != epoch) {
      __nanosleep(32);
      if ((++it & 1023) == 0) {
        if (*((volatile int*)&err->code) != 0 || it > SPIN_LIMIT) {
          if (atomicCAS(&err->code, 0, (int)SFCDD_ERR_TIMEOUT) == 0) err->index = site;
          ok = 0;
          break;
        }
      }
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (ok) (void)ld_acquire(flag);  // every lane acquires the producer's writes
  return ok != 0;
}

// Two consecutive elements of a tile row as the accumulation type.
__device__ __forceinline__ void ld_pair(const double* p, double& a, double& b) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  a = v.x;
  b = v.y;
}
__device__ __forceinline__ void ld_pair(const float* p, float& a, float& b) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  a = v.x;
  b = v.y;
}
__device__ __forceinline__ void ld_pair(const __nv_bfloat16* p, float& a, float& b) {
  const unsigned u = __ldg(reinterpret_cast<const unsigned*>(p));
  a = __uint_as_float(u << 16);
  b = __uint_as_float(u & 0xffff0000u);
}

template <class A>
__device__ __forceinline__ A warp_allsum(A v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Forward row: y_r = Linv_rr (g_r - sum_{c<r} L_rc y_c).
template <class T, class A>
__device__ void fwd_row(const TrsvArgs& a, const T* __restrict__ tiles, int m, int r,
                        double* xs) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long tb = a.ts.tbase[m];
  const int n = a.ts.n[m];
  const int vb = a.ts.vbase[m];
  const int fb = vb / TILE;
  // tile row r is stored contiguously from its first envelope tile kmin to the diagonal
  const int k0 = a.ts.kmin[fb + r];
  const T* row0 = tiles + tb + (long long)a.ts.rowoff[fb + r] * TILE2;  // tile (r, k0)
  A part[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) part[i] = A(0);
  A cur[8][2], nxt[8][2];
  const int ep = reinterpret_cast<const int*>(xs + TILE)[0];
  if (r > k0) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
      ld_pair(row0 + (8 * w + i) * TILE + 2 * lane, cur[i][0], cur[i][1]);
  }
  for (int c = k0; c < r; ++c) {
    if (c + 1 < r) {
      const T* nt_ = row0 + (long long)(c + 1 - k0) * TILE2;
#pragma unroll
      for (int i = 0; i < 8; ++i) ld_pair(nt_ + (8 * w + i) * TILE + 2 * lane, nxt[i][0], nxt[i][1]);
    }
    wait_flag(a.ready + fb + c, ep, a.err, 1);
    const double2 yv = __ldcg(reinterpret_cast<const double2*>(a.y + vb + c * TILE + 2 * lane));
    const A y0 = A(yv.x), y1 = A(yv.y);
    // one fused multiply-add per factor element (FP64 FMA issue rate bounds this loop)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      part[i] = fma(cur[i][0], y0, part[i]);
      part[i] = fma(cur[i][1], y1, part[i]);
    }
    if (c + 1 < r) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        cur[i][0] = nxt[i][0];
        cur[i][1] = nxt[i][1];
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) part[i] = warp_allsum(part[i]);
  if (lane < 8) {
    A mine = A(0);
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (i == lane) mine = part[i];
    const int row = 8 * w + lane;
    const int grow = r * TILE + row;
    double g = 0.0;
    if (grow < n) {
      const MatDesc md = a.md[m];
      if (md.coarse) {
        g = a.g0[md.rhs_base + grow];
      } else {
        int pos = md.start + grow;
        if (pos >= md.rhs_len) pos -= md.rhs_len;
        g = a.rhs[md.rhs_base + pos];
      }
    }
    xs[row] = double(A(g) - mine);
  }
  __syncthreads();
  // diagonal block: y_r = Linv_rr * xs
  const T* dt = row0 + (long long)(r - k0) * TILE2;
  const A x0 = A(xs[2 * lane]), x1 = A(xs[2 * lane + 1]);
  A q[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    A l0, l1;
    ld_pair(dt + (8 * w + i) * TILE + 2 * lane, l0, l1);
    q[i] = fma(l1, x1, l0 * x0);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) q[i] = warp_allsum(q[i]);
  if (lane < 8) {
    A mine = A(0);
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (i == lane) mine = q[i];
    a.y[vb + r * TILE + 8 * w + lane] = double(mine);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) st_release(a.ready + fb + r, ep);
}

// Backward row: d_r = Linv_rr^T (y_r - sum_{c>r} L_cr^T d_c).
template <class T, class A>
__device__ void bwd_row(const TrsvArgs& a, const T* __restrict__ tiles, int m, int r,
                        double* xs, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long tb = a.ts.tbase[m];
  const int nt = a.ts.nt[m];
  const int vb = a.ts.vbase[m];
  const int fb = vb / TILE;
  const int ep = reinterpret_cast<const int*>(xs + TILE)[0];
  A p0 = A(0), p1 = A(0);
  A cur[8][2], nxt[8][2];
  (void)nt;
  // rows c > r whose envelope reaches column r, ascending; consumed from the last
  const int* cl = a.ts.colidx + a.ts.colptr[fb + r];
  const int ncl = a.ts.colptr[fb + r + 1] - a.ts.colptr[fb + r];
  auto tile_ptr = [&](int c) { return tiles + tile_at(a.ts, tb, fb, c, r); };
  if (ncl > 0) {
    const T* t0 = tile_ptr(cl[ncl - 1]);
#pragma unroll
    for (int i = 0; i < 8; ++i) ld_pair(t0 + (8 * w + i) * TILE + 2 * lane, cur[i][0], cur[i][1]);
  }
  for (int q = ncl - 1; q >= 0; --q) {
    const int c = cl[q];
    if (q > 0) {
      const T* t1 = tile_ptr(cl[q - 1]);
#pragma unroll
      for (int i = 0; i < 8; ++i) ld_pair(t1 + (8 * w + i) * TILE + 2 * lane, nxt[i][0], nxt[i][1]);
    }
    wait_flag(a.ready + fb + c, ep, a.err, 2);
    const double* dc = a.dout + vb + c * TILE + 8 * w;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const A dv = A(__ldcg(dc + i));
      p0 += cur[i][0] * dv;
      p1 += cur[i][1] * dv;
    }
    if (q > 0) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        cur[i][0] = nxt[i][0];
        cur[i][1] = nxt[i][1];
      }
    }
  }
  red[w * TILE + 2 * lane] = double(p0);
  red[w * TILE + 2 * lane + 1] = double(p1);
  __syncthreads();
  if (threadIdx.x < TILE) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += red[k * TILE + threadIdx.x];
    // y was written by the forward launch (a previous kernel): plain load is coherent
    xs[threadIdx.x] = double(A(a.y[vb + r * TILE + threadIdx.x]) - A(s));
  }
  __syncthreads();
  const T* dt = tile_ptr(r);
  A q0 = A(0), q1 = A(0);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    A l0, l1;
    ld_pair(dt + (8 * w + i) * TILE + 2 * lane, l0, l1);
    const A xv = A(xs[8 * w + i]);
    q0 += l0 * xv;
    q1 += l1 * xv;
  }
  red[w * TILE + 2 * lane] = double(q0);
  red[w * TILE + 2 * lane + 1] = double(q1);
  __syncthreads();
  if (threadIdx.x < TILE) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += red[k * TILE + threadIdx.x];
    a.dout[vb + r * TILE + threadIdx.x] = double(A(s));
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) st_release(a.ready + fb + r, ep);
}

// Shared layout: xs[TILE] doubles, then the epoch (int) right after.
template <class T, class A, bool FWD>
__global__ void __launch_bounds__(TB) k_trsv(TrsvArgs a) {
  __shared__ double xs[TILE + 1];
  __shared__ double red[8 * TILE];
  __shared__ unsigned long long s_ticket;
  if (threadIdx.x == 0) s_ticket = atomicAdd(a.ticket, 1ull);
  __syncthreads();
  const unsigned long long raw = s_ticket;
  const int t = (int)(raw % (unsigned long long)a.nwork);
  const int epoch = (int)(raw / (unsigned long long)a.nwork) + 1;
  const TrsvWork wk = a.work[t];
  const MatDesc md = a.md[wk.mat];
  if (a.sc && a.sc[md.sub].done) return;
  if (threadIdx.x == 0) reinterpret_cast<int*>(xs + TILE)[0] = epoch;
  __syncthreads();
  if (FWD) {
    if (md.coarse)
      fwd_row<double, double>(a, a.ctiles, wk.mat, wk.row, xs);
    else
      fwd_row<T, A>(a, reinterpret_cast<const T*>(a.ltiles), wk.mat, wk.row, xs);
  } else {
    if (md.coarse)
      bwd_row<double, double>(a, a.ctiles, wk.mat, wk.row, xs, red);
    else
      bwd_row<T, A>(a, reinterpret_cast<const T*>(a.ltiles), wk.mat, wk.row, xs, red);
  }
}

void launch_trsv_fwd(const TrsvArgs& a, Store st, cudaStream_t s) {
  switch (st) {
    case Store::F64: k_trsv<double, double, true><<<a.nwork, TB, 0, s>>>(a); break;
    case Store::F32: k_trsv<float, float, true><<<a.nwork, TB, 0, s>>>(a); break;
    default: k_trsv<__nv_bfloat16, float, true><<<a.nwork, TB, 0, s>>>(a); break;
  }
}

void launch_trsv_bwd(const TrsvArgs& a, Store st, cudaStream_t s) {
  switch (st) {
    case Store::F64: k_trsv<double, double, false><<<a.nwork, TB, 0, s>>>(a); break;
    case Store::F32: k_trsv<float, float, false><<<a.nwork, TB, 0, s>>>(a); break;
    default: k_trsv<__nv_bfloat16, float, false><<<a.nwork, TB, 0, s>>>(a); break;
  }
}

}  // namespace sfcdd
