// Setup-phase matrices and their factorization.
//
// Local matrices A_i = R_i A R_i^T (Sec. 3.1; Algorithm 1, steps 6-7): the
// principal submatrix of the stencil operator on the curve positions of
// Omega_i, assembled tile by tile straight from the curve (no CRS copy).
// Coarse matrix A_0 = R_0 A R_0^T (eq. csm; Algorithm 1, step 10): entry (a, b)
// is [a = b] |a| diag - sum_j w_j E_j(a, b), where E_j counts the axis-j
// neighbour pairs (u in block a, v in block b); the integer counts make the
// assembly exact and deterministic.
// Factorization (Sec. 3.1: factor once, then only forward/backward solves): a
// blocked right-looking Cholesky on TILE x TILE tiles, batched over all
// matrices.  Only tiles inside the Cholesky envelope are stored and updated:
// row r of the factor is zero left of the first nonzero of row r of A, so the
// tiles left of a tile row's envelope stay exact zeros and skipping them gives
// the same factor.  Per step k one launch factors the diagonal tiles (and
// inverts the factor's diagonal block in place), one solves the panel tiles of
// column k, one updates the trailing tiles they touch.
#include <algorithm>

#include "device_common.cuh"
#include "oz_tile.cuh"
#include "tc_tile.cuh"

namespace sfcdd {

constexpr int FB = 256;

template <class T>
__device__ __forceinline__ T from_double(double v) { return T(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_double<__nv_bfloat16>(double v) {
  return __float2bfloat16_rn((float)v);
}

// ---------------------------------------------------------------------------
// Envelopes.
__global__ void k_envelope_init(TileSetDev ts, int nmat, int* tfirst) {
  const int m = grid_mat();
  if (m >= nmat) return;
  const int nt = ts.nt[m];
  const int fb = ts.vbase[m] / TILE;
  for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nt; I += gridDim.x * blockDim.x)
    tfirst[fb + I] = I * TILE;  // the diagonal
}

void launch_envelope_init(const TileSetDev& ts, int nmat, int max_nt, int* tfirst, cudaStream_t s) {
  k_envelope_init<<<mat_grid((max_nt + 127) / 128, nmat), 128, 0, s>>>(ts, nmat, tfirst);
}

// Row r of A_i: smallest local column among its neighbours inside Omega_i.
__global__ void k_envelope_local(GridDev g, PartDev pd, const unsigned* __restrict__ code,
                                 const int* __restrict__ invpad, TileSetDev ts, int nmat,
                                 int* tfirst) {
  const int m = grid_mat();
  if (m >= nmat) return;
  const int n = ts.n[m];
  const int fb = ts.vbase[m] / TILE;
  const int start = pd.start[m];
  const int vb = ts.vbase[m];
  const LocalOrder lo{ts.lperm ? ts.lperm + vb : nullptr, ts.linv ? ts.linv + vb : nullptr};
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const int first = envelope_row(g, code, invpad, start, n, lo, r);
    if (first < r) atomicMin(&tfirst[fb + r / TILE], first);
  }
}

void launch_envelope_local(const GridDev& g, const PartDev& pd, const unsigned* code,
                           const int* invpad, const TileSetDev& ts, int nmat, int max_n, int* tfirst,
                           cudaStream_t s) {
  k_envelope_local<<<mat_grid((max_n + 255) / 256, nmat), 256, 0, s>>>(g, pd, code, invpad, ts,
                                                                      nmat, tfirst);
}

// Coarse row a: smallest coarse row adjacent to row a (factor numbering).
__global__ void k_envelope_coarse(GridDev g, PartDev pd, const unsigned* __restrict__ code,
                                  const int* __restrict__ invpad, int fbc, int* tfirst) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < g.N; p += gridDim.x * blockDim.x) {
    int a;
    const int first = envelope_coarse_point(g, pd, code, invpad, p, a);
    if (first < a) atomicMin(&tfirst[fbc + a / TILE], first);
  }
}

void launch_envelope_coarse(const GridDev& g, const PartDev& pd, const unsigned* code,
                            const int* invpad, int fb_coarse, int* tfirst, cudaStream_t s) {
  const int nb = min((g.N + 255) / 256, 152 * 8);
  k_envelope_coarse<<<nb, 256, 0, s>>>(g, pd, code, invpad, fb_coarse, tfirst);
}

// ---------------------------------------------------------------------------
// Local matrices.  grid = (max stored tiles per matrix, nmat); one CTA per tile.
template <class T>
__global__ void __launch_bounds__(FB) k_assemble_local(GridDev g, PartDev pd,
                                                       const unsigned* __restrict__ code,
                                                       const int* __restrict__ invpad,
                                                       TileSetDev ts, int mat0, int nmat,
                                                       T* __restrict__ tiles) {
  __shared__ double sm[TILE2];
  if (grid_mat() >= nmat) return;
  const int m = mat0 + grid_mat();
  const int nt = ts.nt[m];
  const int fb = ts.vbase[m] / TILE;
  const int idx = blockIdx.x;
  if (idx >= stored_tiles(ts, fb, nt)) return;
  int a, b;
  skyline_decode(ts, fb, nt, idx, a, b);
  for (int k = threadIdx.x; k < TILE2; k += FB) sm[k] = 0.0;
  __syncthreads();
  const int vb = ts.vbase[m];
  const LocalOrder lo{ts.lperm ? ts.lperm + vb : nullptr, ts.linv ? ts.linv + vb : nullptr};
  assemble_local_tile(g, code, invpad, pd.start[m], ts.n[m], lo, a, b, sm);
  __syncthreads();
  T* out = tiles + ts.tbase[m] + (long long)idx * TILE2;
  for (int k = threadIdx.x; k < TILE2; k += FB) out[k] = from_double<T>(sm[k]);
}

void launch_assemble_local(const GridDev& g, const PartDev& pd, const unsigned* code,
                           const int* invpad, const TileSetDev& ts, int mat0, int nmat, int max_tiles,
                           void* tiles, Store st, cudaStream_t s) {
  const dim3 grid = mat_grid(max_tiles, nmat);
  switch (st) {
    case Store::F64:
      k_assemble_local<double><<<grid, FB, 0, s>>>(g, pd, code, invpad, ts, mat0, nmat, (double*)tiles);
      break;
    case Store::F32:
      k_assemble_local<float><<<grid, FB, 0, s>>>(g, pd, code, invpad, ts, mat0, nmat, (float*)tiles);
      break;
    default:
      k_assemble_local<__nv_bfloat16><<<grid, FB, 0, s>>>(g, pd, code, invpad, ts, mat0, nmat,
                                                          (__nv_bfloat16*)tiles);
      break;
  }
}

// ---------------------------------------------------------------------------
// Coarse matrix tiles (a one-matrix tile set).  One CTA per stored tile;
// 4 threads per coarse row walk the points of the row's block.
__global__ void __launch_bounds__(FB) k_assemble_coarse(GridDev g, PartDev pd,
                                                        const unsigned* __restrict__ code,
                                                        const int* __restrict__ invpad,
                                                        TileSetDev cts, double* __restrict__ tiles) {
  extern __shared__ __align__(16) unsigned char dsm_coarse[];
  double* acc = reinterpret_cast<double*>(dsm_coarse);
  int* cnt = reinterpret_cast<int*>(acc + TILE2);
  const int nt = cts.nt[0];
  const int fb = cts.vbase[0] / TILE;
  int R, C;
  skyline_decode(cts, fb, nt, blockIdx.x, R, C);
  assemble_coarse_tile(g, pd, cts.n[0], code, invpad, R, C, acc, cnt);
  double* out = tiles + cts.tbase[0] + (long long)blockIdx.x * TILE2;
  for (int k = threadIdx.x; k < TILE2; k += FB) out[k] = acc[k];
}

void launch_assemble_coarse(const GridDev& g, const PartDev& pd, const unsigned* code,
                            const int* invpad, const TileSetDev& cts, int ntiles, double* tiles,
                            cudaStream_t s) {
  const int smem = TILE2 * (int)(sizeof(double) + sizeof(int));
  cudaFuncSetAttribute(k_assemble_coarse, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_assemble_coarse<<<ntiles, FB, smem, s>>>(g, pd, code, invpad, cts, tiles);
}

// ---------------------------------------------------------------------------
// Factorization kernels, compute type T (double or float), storage T.

// Diagonal tile k of every matrix with nt > k: Cholesky of the tile, then the
// inverse of its lower-triangular factor replaces it.  Two algorithms, one per
// compute type, chosen by what bounds each on this part:
//   FP64 (potrf_tile_column): a warp's FP64 instruction occupies its
//   sub-partition's FP64 unit for about 64 cycles whatever its predicate, so
//   the work is laid out for few issued FP64 instructions and a short
//   dependent chain: the factorization and the inverse advance together one
//   column per iteration, every entry of the lower triangle held in one
//   thread's registers, and an instruction issues only where some lane of the
//   warp still has a live entry.
//   FP32 (potrf_tile_blocked): FP32 issue is cheap and the blocked algorithm's
//   16-wide products keep all eight warps busy with fewer barriers.
// Both read the tile through L2 (it may have been written by other CTAs of the
// same launch, after a fence) and use dsm, 2 (TILE + 1)^2 elements of T.
// rows: the tile's rows inside the matrix (the last tile of a matrix whose size
// is not a multiple of TILE); the rows beyond are identity padding with zero
// couplings, the identity in L and in L^{-1}, so only the matrix rows are
// factored.
constexpr int PB = 16;           // column block of the blocked algorithm
constexpr int PNB = TILE / PB;   // blocks per tile

__device__ __forceinline__ void potrf_bar128() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// lower-triangle index e -> (i, l), i >= l
__device__ __forceinline__ void tri_rc(int e, int& i, int& l) {
  int t = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while ((t + 1) * (t + 2) / 2 <= e) ++t;
  while (t * (t + 1) / 2 > e) --t;
  i = t;
  l = e - t * (t + 1) / 2;
}

template <class T>
__device__ void potrf_tile(T* __restrict__ tp, unsigned char* dsm, ErrWord* err, int m,
                           int rows = TILE);

// Rows of matrix m inside its diagonal tile k.
__device__ __forceinline__ int tile_rows(const TileSetDev& ts, int m, int k) {
  return min(TILE, ts.n[m] - k * TILE);
}

// A non-positive pivot marks matrix m not SPD (first error wins) and continues
// with 1 so that the kernel finishes; returns 1 / sqrt(pivot).
template <class T>
__device__ __forceinline__ T pivot_rsqrt(T d, ErrWord* err, int m) {
  if (!(d > T(0))) {
    if (atomicCAS(&err->code, 0, (int)SFCDD_ERR_NOT_SPD) == 0) err->index = m;
    d = T(1);
  }
  return rsqrt(d);
}

// Blocked right-looking Cholesky with 16-column blocks:
//   per block b: warps 0-3 factor the 16 x 16 diagonal block D_b (one element
//   of its triangle per thread, reciprocal pivots, scaling applied once at the
//   end) and invert it into X (row by row, 8 threads per dot product); then
//   all warps form the panel L_pb = A_pb D_b^{-T} and update the trailing
//   triangle with it.
// The off-diagonal 16 x 16 blocks of X = L^{-1} follow by diagonals:
// X_ab = -X_aa sum_{k=b}^{a-1} L_ak X_kb.  Padding rows fill whole 16-column
// blocks, which are left out.
template <class T>
__device__ void potrf_tile_blocked(T* __restrict__ tp, unsigned char* dsm, ErrWord* err, int m,
                                   int rows) {
  T (*L)[TILE + 1] = reinterpret_cast<T (*)[TILE + 1]>(dsm);
  T (*X)[TILE + 1] = L + TILE;
  T* rinv = &X[TILE][0];  // TILE reciprocal pivots (row TILE of X, TILE + 1 entries)
  const int tid = threadIdx.x;
  for (int e = tid; e < TILE2; e += FB) L[e / TILE][e % TILE] = __ldcg(tp + e);
  for (int e = tid; e < TILE2; e += FB) X[e / TILE][e % TILE] = T(0);
  // my elements of a 16 x 16 lower triangle (136 of them; threads < 128)
  int di0 = 0, dl0 = 0, di1 = -1, dl1 = -1;
  if (tid < 128) {
    tri_rc(tid, di0, dl0);
    if (tid + 128 < PB * (PB + 1) / 2) tri_rc(tid + 128, di1, dl1);
  }
  __syncthreads();
  const int nbr = rows >= TILE ? PNB : (rows + PB - 1) / PB;  // blocks with matrix rows
  const int rtop = PB * nbr;
  for (int b = 0; b < nbr; ++b) {
    const int o = PB * b;
    if (tid < 128) {
      // factor D_b in place (column scaling deferred): d_c -> rinv, trailing update
      for (int c = 0; c < PB; ++c) {
        T d = L[o + c][o + c];
        if (!(d > T(0))) {
          if (tid == 0 && atomicCAS(&err->code, 0, (int)SFCDD_ERR_NOT_SPD) == 0) err->index = m;
          d = T(1);
        }
        const T r = rsqrt(d);
        const T dinv = r * r;
        if (tid == 0) rinv[o + c] = r;
        if (dl0 > c) L[o + di0][o + dl0] -= L[o + di0][o + c] * (L[o + dl0][o + c] * dinv);
        if (dl1 > c) L[o + di1][o + dl1] -= L[o + di1][o + c] * (L[o + dl1][o + c] * dinv);
        potrf_bar128();
      }
      // deferred scaling of the strictly lower part
      if (di0 > dl0) L[o + di0][o + dl0] *= rinv[o + dl0];
      if (di1 > dl1) L[o + di1][o + dl1] *= rinv[o + dl1];
      potrf_bar128();
      // D_b^{-1}: row i needs rows < i; column c = tid / 8, eight threads per dot
      const int c = tid >> 3, part = tid & 7;
      for (int i = 0; i < PB; ++i) {
        T sacc = T(0);
        if (c < i)
          for (int kk = c + part; kk < i; kk += 8) sacc += L[o + i][o + kk] * X[o + kk][o + c];
        sacc += __shfl_xor_sync(0xffffffffu, sacc, 1);
        sacc += __shfl_xor_sync(0xffffffffu, sacc, 2);
        sacc += __shfl_xor_sync(0xffffffffu, sacc, 4);
        if (part == 0 && c <= i) X[o + i][o + c] = c == i ? rinv[o + i] : -sacc * rinv[o + i];
        potrf_bar128();
      }
    }
    __syncthreads();
    const int o2 = o + PB, rest = rtop - o2;  // matrix rows below the block
    if (rest > 0) {
      // panel L_pc = sum_{k <= c} A_pk X_ck  (D^{-T} is X^T), written after all reads
      T pv[3];
      int np = 0;
      for (int e = tid; e < rest * PB; e += FB, ++np) {
        const int p = o2 + e / PB, cc = e % PB;
        T acc = T(0);
        for (int kk = 0; kk <= cc; ++kk) acc += L[p][o + kk] * X[o + cc][o + kk];
        pv[np] = acc;
      }
      __syncthreads();
      np = 0;
      for (int e = tid; e < rest * PB; e += FB, ++np) L[o2 + e / PB][o + e % PB] = pv[np];
      __syncthreads();
      // trailing triangle A_pq -= sum_k L_pk L_qk (p >= q >= o2)
      for (int e = tid; e < rest * (rest + 1) / 2; e += FB) {
        int pi, qi;
        tri_rc(e, pi, qi);
        const int p = o2 + pi, q = o2 + qi;
        T acc = T(0);
#pragma unroll
        for (int kk = 0; kk < PB; ++kk) acc += L[p][o + kk] * L[q][o + kk];
        L[p][q] -= acc;
      }
      __syncthreads();
    }
  }
  // off-diagonal blocks of X by diagonals d = a - b; S_ab is staged in the
  // (zero) upper block (b, a) of X
  for (int d = 1; d < nbr; ++d) {
    const int nblk = nbr - d;
    for (int e = tid; e < nblk * PB * PB; e += FB) {
      const int bb = e / (PB * PB), a = bb + d;
      const int i = (e / PB) % PB, j = e % PB;
      T acc = T(0);
      for (int k = bb; k < a; ++k)
        for (int kk = 0; kk < PB; ++kk) acc += L[PB * a + i][PB * k + kk] * X[PB * k + kk][PB * bb + j];
      X[PB * bb + i][PB * a + j] = acc;  // S_ab into the upper block (b, a)
    }
    __syncthreads();
    for (int e = tid; e < nblk * PB * PB; e += FB) {
      const int bb = e / (PB * PB), a = bb + d;
      const int i = (e / PB) % PB, j = e % PB;
      T acc = T(0);
      for (int kk = 0; kk <= i; ++kk) acc += X[PB * a + i][PB * a + kk] * X[PB * bb + kk][PB * a + j];
      X[PB * a + i][PB * bb + j] = -acc;
    }
    __syncthreads();
  }
  for (int e = tid; e < TILE2; e += FB) {
    const int r = e / TILE, c = e % TILE;
    tp[e] = c > r ? T(0) : (r >= rtop ? (r == c ? T(1) : T(0)) : X[r][c]);
  }
}

// Right-looking Cholesky fused with the row-oriented inverse X = L^{-1}, one
// column per iteration k.  Warp 0 owns the diagonal, takes the pivots'
// reciprocal square roots and scales what is published; warps 1-7 own the
// 2016 entries below the diagonal, 9 each, in registers.  An entry is L(i, j)
// until column j is final and from then on Y(i, j), the open part of row i of
// X, which starts at zero (Y starts as the identity).  Iteration k:
//   A (warp 0): r_k = 1 / sqrt(pivot k); L(i, k) = raw(i, k) r_k for i > k and
//      X(k, j) = Y(k, j) r_k for j < k, X(k, k) = r_k, into shared memory; row
//      k of X is final and goes to the tile.
//   B (all): L(i, j) -= L(i, k) L(j, k) for k < j <= i and
//      Y(i, j) -= L(i, k) X(k, j) for j <= k < i; the entries that become
//      column k + 1 or row k + 1 publish their raw values; warp 0 finishes
//      pivot k + 1 and inverts it.
// A slot is skipped by the whole warp when none of its lanes holds a live
// entry (rows above k or in the padding), which saves the FP64 issue of the
// triangle's shrinking part; the scaling costs one multiplication per
// published value.
template <class T>
__device__ void potrf_tile_column(T* __restrict__ tp, unsigned char* dsm, ErrWord* err, int m,
                                  int rows) {
  constexpr int NE = FB - 32;                                // threads owning entries
  constexpr int NS = (TILE * (TILE - 1) / 2 + NE - 1) / NE;  // entries per thread
  T* colbuf = reinterpret_cast<T*>(dsm);  // L(:, k), scaled
  T* rowbuf = colbuf + TILE;              // X(k, :)
  T* colraw = rowbuf + TILE;              // L(:, k + 1) before scaling
  T* rowraw = colraw + TILE;              // Y(k + 1, :) before scaling
  T* rinv = rowraw + TILE;                // reciprocal pivots
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int n = rows < TILE ? rows : TILE;  // matrix rows; the rest is identity padding
  T v[NS];
  int ii[NS], jj[NS];
  T dg[2] = {T(0), T(0)};
  if (w == 0) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = lane + 32 * h;
      dg[h] = __ldcg(tp + i * TILE + i);
    }
  } else {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const int e = tid - 32 + NE * s;
      if (e < TILE * (TILE - 1) / 2) {
        int a, b;
        tri_rc(e, a, b);  // strictly lower entry: row a + 1, column b
        ii[s] = a + 1;
        jj[s] = b;
        v[s] = __ldcg(tp + ii[s] * TILE + jj[s]);
        if (jj[s] == 0 && ii[s] < n) colraw[ii[s]] = v[s];  // column 0 is final as loaded
      } else {
        ii[s] = 0;  // no entry: never live
        jj[s] = 0;
        v[s] = T(0);
      }
    }
  }
  __syncthreads();  // every entry is in registers: the tile may be overwritten
  if (tid == 0) rinv[0] = pivot_rsqrt(dg[0], err, m);
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (w == 0) {
      const T r = rinv[k];
      for (int i = k + 1 + lane; i < n; i += 32) colbuf[i] = colraw[i] * r;
      for (int j = lane; j < k; j += 32) {
        const T x = rowraw[j] * r;
        rowbuf[j] = x;
        tp[k * TILE + j] = x;
      }
      if (lane == 0) {
        rowbuf[k] = r;
        tp[k * TILE + k] = r;
      }
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        const bool live = i > k && i < n;
        if (__any_sync(0xffffffffu, live) && live) {
          const T l = colbuf[i];
          dg[h] -= l * l;
          if (i == k + 1) rinv[k + 1] = pivot_rsqrt(dg[h], err, m);
        }
      }
    } else {
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const int i = ii[s], j = jj[s];
        const bool live = i > k && i < n;
        if (__any_sync(0xffffffffu, live) && live) {
          // L(i, j) while j > k; at j == k it turns into Y(i, k) = 0 - L(i, k) X(k, k)
          const T b = j > k ? colbuf[j] : rowbuf[j];
          const T base = j == k ? T(0) : v[s];
          v[s] = base - colbuf[i] * b;
          if (j == k + 1) colraw[i] = v[s];       // column k + 1 is final
          else if (i == k + 1) rowraw[j] = v[s];  // row k + 1 of Y is final
        }
      }
    }
    __syncthreads();
  }
  // above the diagonal zeros, the padding rows the identity
  for (int e = tid; e < TILE2; e += FB) {
    const int rr = e / TILE, c = e % TILE;
    if (c > rr) tp[e] = T(0);
    else if (rr >= n) tp[e] = rr == c ? T(1) : T(0);
  }
}

template <class T>
__device__ void potrf_tile(T* __restrict__ tp, unsigned char* dsm, ErrWord* err, int m, int rows) {
  if constexpr (sizeof(T) == 8) potrf_tile_column<T>(tp, dsm, err, m, rows);
  else potrf_tile_blocked<T>(tp, dsm, err, m, rows);
}

__global__ void __launch_bounds__(FB) k_potrf_one(double* tile, ErrWord* err, int m) {
  extern __shared__ __align__(16) unsigned char dsm_one[];
  potrf_tile<double>(tile, dsm_one, err, m);
}

void launch_potrf_one(double* tile, ErrWord* err, int m, cudaStream_t s) {
  const int smem = (2 * TILE + 1) * (TILE + 1) * (int)sizeof(double);
  cudaFuncSetAttribute(k_potrf_one, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_potrf_one<<<1, FB, smem, s>>>(tile, err, m);
}

template <class T>
__global__ void __launch_bounds__(FB) k_potrf(TileSetDev ts, int mat0, int k, T* __restrict__ tiles,
                                              ErrWord* err) {
  extern __shared__ __align__(16) unsigned char dsm_potrf[];
  const int m = mat0 + blockIdx.x;
  if (ts.nt[m] <= k) return;
  const int fb = ts.vbase[m] / TILE;
  potrf_tile<T>(tiles + tile_at(ts, ts.tbase[m], fb, k, k), dsm_potrf, err, m, tile_rows(ts, m, k));
}

// C = X * Y^T on 64x64 tiles (X, Y row-major in global), each thread a 4x4 block.
// Shared tiles are stored transposed so the k-loop reads contiguous vectors.
template <class T>
__device__ __forceinline__ void load_transposed(T (*dst)[TILE + 4], const T* __restrict__ src) {
  for (int e = threadIdx.x; e < TILE2; e += FB) dst[e % TILE][e / TILE] = src[e];
}

template <class T>
__device__ __forceinline__ void mma_4x4(T (&acc)[4][4], T (*Xt)[TILE + 4], T (*Yt)[TILE + 4],
                                        int r0, int c0) {
#pragma unroll 8
  for (int s = 0; s < TILE; ++s) {
    T xv[4], yv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      xv[i] = Xt[s][r0 + i];
      yv[i] = Yt[s][c0 + i];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) acc[i][jj] += xv[i] * yv[jj];
  }
}

// Rows [r_lo, r_lo + n) of a row-major tile into columns of a transposed
// shared array (dst[s][r] = src[r][s]).
template <class T>
__device__ __forceinline__ void load_rows_transposed(T (*dst)[TILE + 4], const T* __restrict__ src,
                                                     int r_lo, int n) {
  for (int e = threadIdx.x; e < n * TILE; e += FB) {
    const int r = r_lo + e / TILE, c = e % TILE;
    dst[c][r] = src[r * TILE + c];
  }
}

// Output rows of one CTA of a tile product X Y^T: with SPLIT = 1 the whole tile,
// each thread a 4 x 4 block; with SPLIT = 4 a 16-row slab (rows 16 slab ..),
// each thread 1 x 4.  Splitting puts the FP64 work of one tile on four SMs.
template <int SPLIT>
struct SlabMap {
  static constexpr int RA = 4 / SPLIT;  // rows per thread
  int r0, c0;
  __device__ SlabMap(int slab) {
    if (SPLIT == 1) {
      r0 = (threadIdx.x / 16) * 4;
    } else {
      r0 = 16 * slab + threadIdx.x / 16;
    }
    c0 = (threadIdx.x % 16) * 4;
  }
};

template <class T, int RA>
__device__ __forceinline__ void mma_rows(T (&acc)[RA][4], T (*Xt)[TILE + 4], T (*Yt)[TILE + 4],
                                         int r0, int c0) {
#pragma unroll 8
  for (int s = 0; s < TILE; ++s) {
    T xv[RA], yv[4];
#pragma unroll
    for (int i = 0; i < RA; ++i) xv[i] = Xt[s][r0 + i];
#pragma unroll
    for (int i = 0; i < 4; ++i) yv[i] = Yt[s][c0 + i];
#pragma unroll
    for (int i = 0; i < RA; ++i)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) acc[i][jj] += xv[i] * yv[jj];
  }
}

// Panel: L_ik = A_ik * Linv_kk^T for the stored tiles of column k below the
// diagonal.  grid = (max panel rows * SPLIT, nmat); a CTA reads and writes
// only the rows of its slab of A_ik.
template <class T, int SPLIT>
__global__ void __launch_bounds__(FB) k_trsm(TileSetDev ts, int mat0, int nmat, int k,
                                             T* __restrict__ tiles) {
  extern __shared__ __align__(16) unsigned char dsm_trsm[];
  T (*At)[TILE + 4] = reinterpret_cast<T (*)[TILE + 4]>(dsm_trsm);
  T (*Bt)[TILE + 4] = At + TILE;
  if (grid_mat() >= nmat) return;
  const int m = mat0 + grid_mat();
  const int nt = ts.nt[m];
  if (k >= nt) return;
  const int fb = ts.vbase[m] / TILE;
  const int c0p = ts.colptr[fb + k];
  const int tix = blockIdx.x / SPLIT, slab = blockIdx.x % SPLIT;
  if (tix >= ts.colptr[fb + k + 1] - c0p) return;
  const int i = ts.colidx[c0p + tix];
  const long long tb = ts.tbase[m];
  T* aik = tiles + tile_at(ts, tb, fb, i, k);
  const T* lkk = tiles + tile_at(ts, tb, fb, k, k);
  load_rows_transposed<T>(At, aik, (TILE / SPLIT) * slab, TILE / SPLIT);
  load_transposed<T>(Bt, lkk);
  __syncthreads();
  const SlabMap<SPLIT> mp(slab);
  constexpr int RA = SlabMap<SPLIT>::RA;
  T acc[RA][4];
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  mma_rows<T, RA>(acc, At, Bt, mp.r0, mp.c0);
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) aik[(mp.r0 + a) * TILE + mp.c0 + b] = acc[a][b];
}

// Trailing update A_ij -= L_ik L_jk^T for the stored panel tiles i >= j of
// column k, and the factorization of diagonal tile k+1 (step k+1's potrf) as
// soon as its last update is in: the last of the SPLIT CTAs updating tile
// (k+1, k+1) (counted in diag_cnt[fb + k + 1], zero before the factorization)
// factors it, or, when column k does not reach row k+1, the launch's last CTA
// does.  grid = (max pairs * SPLIT + 1, nmat)
template <class T, int SPLIT>
__global__ void __launch_bounds__(FB) k_syrk(TileSetDev ts, int mat0, int nmat, int k,
                                             T* __restrict__ tiles,
                                             int* __restrict__ diag_cnt, ErrWord* err) {
  extern __shared__ __align__(16) unsigned char dsm_syrk[];
  T (*Xt)[TILE + 4] = reinterpret_cast<T (*)[TILE + 4]>(dsm_syrk);
  T (*Yt)[TILE + 4] = Xt + TILE;
  __shared__ int s_last;
  if (grid_mat() >= nmat) return;
  const int m = mat0 + grid_mat();
  const int nt = ts.nt[m];
  if (k >= nt) return;
  const int fb = ts.vbase[m] / TILE;
  const int c0p = ts.colptr[fb + k];
  const int cnt = ts.colptr[fb + k + 1] - c0p;
  const long long tb = ts.tbase[m];
  if ((int)blockIdx.x == (int)gridDim.x - 1) {
    // column k does not reach row k+1: tile (k+1, k+1) is final already
    if (k + 1 < nt && ts.kmin[fb + k + 1] > k)
      potrf_tile<T>(tiles + tile_at(ts, tb, fb, k + 1, k + 1), dsm_syrk, err, m,
                    tile_rows(ts, m, k + 1));
    return;
  }
  const int tix = blockIdx.x / SPLIT, slab = blockIdx.x % SPLIT;
  if (tix >= cnt * (cnt + 1) / 2) return;
  int ii, jj;
  tri_decode(tix, ii, jj);
  const int i = ts.colidx[c0p + ii], j = ts.colidx[c0p + jj];
  const T* lik = tiles + tile_at(ts, tb, fb, i, k);
  const T* ljk = tiles + tile_at(ts, tb, fb, j, k);
  T* aij = tiles + tile_at(ts, tb, fb, i, j);
  load_rows_transposed<T>(Xt, lik, (TILE / SPLIT) * slab, TILE / SPLIT);
  load_transposed<T>(Yt, ljk);
  __syncthreads();
  const SlabMap<SPLIT> mp(slab);
  constexpr int RA = SlabMap<SPLIT>::RA;
  T acc[RA][4];
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  mma_rows<T, RA>(acc, Xt, Yt, mp.r0, mp.c0);
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) aij[(mp.r0 + a) * TILE + mp.c0 + b] -= acc[a][b];
  if (i == k + 1 && j == k + 1) {
    __threadfence();
    __syncthreads();  // every slab row of this CTA is written (and the smem reads done)
    if (threadIdx.x == 0) s_last = atomicAdd(&diag_cnt[fb + k + 1], 1) == SPLIT - 1;
    __syncthreads();
    if (s_last) {
      __threadfence();
      potrf_tile<T>(aij, dsm_syrk, err, m, tile_rows(ts, m, k + 1));
    }
  }
}

// ---------------------------------------------------------------------------
// FP32 panel and trailing update on the tensor cores (tcgen05, FP32 accumulation
// in tensor memory).  One CTA computes two tile products that share their right
// operand as one M = 128 MMA chain: rows 0-63 of A are the first tile, rows
// 64-127 the second (or the first again when there is no second).
// BF = false: TF32 operands with the error-compensated hi/lo split (see
// tc_tile.cuh), FP32-accurate products.  BF = true: the operands rounded to
// bf16 (one kind::f16 MMA per K = 16 step), the BF16 factorization: bf16
// operands, FP32 accumulation, FP32 working tiles and diagonal factorizations.

// Stage rows [row0, row0 + 64) of a bf16 operand from a row-major 64 x 64 FP32
// tile, rounded to nearest: 8 consecutive columns form one 16-byte core row
// (the K-major layout of oz_tile.cuh: LBO 128, SBO 1024).
__device__ __forceinline__ void stage_tile_bf16(unsigned char* dst, const float* __restrict__ src,
                                                int row0) {
  for (int e = threadIdx.x; e < 64 * 8; e += blockDim.x) {
    const int r = e >> 3, c8 = e & 7;
    const float4 v0 = *reinterpret_cast<const float4*>(src + r * 64 + 8 * c8);
    const float4 v1 = *reinterpret_cast<const float4*>(src + r * 64 + 8 * c8 + 4);
    auto pack = [](float lo, float hi) {
      const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);  // lo in the low half
      return *reinterpret_cast<const uint32_t*>(&b);
    };
    const uint4 w = make_uint4(pack(v0.x, v0.y), pack(v0.z, v0.w), pack(v1.x, v1.y),
                               pack(v1.z, v1.w));
    *reinterpret_cast<uint4*>(dst + oz::core_offset(row0 + r, c8)) = w;
  }
}

// Shared memory of one product: TF32 split A_hi | A_lo | B_hi | B_lo, bf16 A | B;
// then the mbarrier and the tensor-memory address.
template <bool BF>
__host__ __device__ constexpr uint32_t tc_operand_bytes() {
  return BF ? oz::A_SLICE + oz::B_SLICE : 2 * tc::A_BYTES + 2 * tc::B_BYTES;
}
template <bool BF>
__host__ __device__ constexpr int tc_smem_bytes() {
  return (int)tc_operand_bytes<BF>() + 16;
}

// Stage, multiply, and hand each thread its 32 accumulator columns; returns
// false (error word set) when the MMA completion wait ran out.
template <bool BF>
__device__ __forceinline__ bool tc_product(unsigned char* dsm, const float* a0, const float* a1,
                                           const float* b, float (&v)[32], int& row, int& col0,
                                           uint32_t& tmem, ErrWord* err, int m) {
  using namespace tc;
  uint64_t* bar = reinterpret_cast<uint64_t*>(dsm + tc_operand_bytes<BF>());
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  if (threadIdx.x < 32) tmem_alloc(tslot);
  if (threadIdx.x == 0) {
    mbar_init1(bar);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if constexpr (BF) {
    stage_tile_bf16(dsm, a0, 0);
    stage_tile_bf16(dsm, a1, 64);
    stage_tile_bf16(dsm + oz::A_SLICE, b, 0);
  } else {
    unsigned char* ahi = dsm;
    unsigned char* alo = dsm + A_BYTES;
    unsigned char* bhi = dsm + 2 * A_BYTES;
    unsigned char* blo = bhi + B_BYTES;
    stage_tile(ahi, alo, a0, 0);
    stage_tile(ahi, alo, a1, 64);
    stage_tile(bhi, blo, b, 0);
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  tmem = *tslot;
  if (threadIdx.x == 0) {
    if constexpr (BF) {
      const uint32_t a = smem_addr(dsm), bb = smem_addr(dsm + oz::A_SLICE);
#pragma unroll
      for (int kk = 0; kk < TC_K / 16; ++kk) {
        const uint32_t o = (uint32_t)kk * 2 * oz::LBO;
        oz::mma_bf16(tmem, oz::make_desc(a + o), oz::make_desc(bb + o), kk > 0 ? 1u : 0u);
      }
    } else {
      issue_product(tmem, dsm, dsm + A_BYTES, dsm + 2 * A_BYTES, dsm + 2 * A_BYTES + B_BYTES);
    }
    mma_commit(bar);
  }
  const bool ok = mbar_wait_bounded(bar, 0, 1ll << 24);
  fence_after_sync();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  row = 32 * (w & 3) + lane;
  col0 = 32 * (w >> 2);
  if (ok) {
    tmem_ld32(tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)col0, v);
  } else if (lane == 0 && atomicCAS(&err->code, 0, (int)SFCDD_ERR_TIMEOUT) == 0) {
    err->index = m;
  }
  return ok;
}

// Every thread is done with its tensor-memory reads: release the columns.
__device__ __forceinline__ void tc_release(uint32_t tmem) {
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) tc::tmem_dealloc(tmem);
}

// Panel L_ik = A_ik Linv_kk^T, two stored tiles of column k per CTA.
// grid = (ceil(max panel rows / 2), nmat)
template <bool BF>
__global__ void __launch_bounds__(FB) k_trsm_tc(TileSetDev ts, int mat0, int nmat, int k,
                                                float* __restrict__ tiles, ErrWord* err) {
  extern __shared__ __align__(1024) unsigned char dsm_tc[];
  if (grid_mat() >= nmat) return;
  const int m = mat0 + grid_mat();
  const int nt = ts.nt[m];
  if (k >= nt) return;
  const int fb = ts.vbase[m] / TILE;
  const int c0p = ts.colptr[fb + k];
  const int cnt = ts.colptr[fb + k + 1] - c0p;
  const int t0 = 2 * (int)blockIdx.x;
  if (t0 >= cnt) return;
  const bool two = t0 + 1 < cnt;
  const long long tb = ts.tbase[m];
  float* a0 = tiles + tile_at(ts, tb, fb, ts.colidx[c0p + t0], k);
  float* a1 = two ? tiles + tile_at(ts, tb, fb, ts.colidx[c0p + t0 + 1], k) : a0;
  const float* lkk = tiles + tile_at(ts, tb, fb, k, k);
  float v[32];
  int row, col0;
  uint32_t tmem;
  const bool ok = tc_product<BF>(dsm_tc, a0, a1, lkk, v, row, col0, tmem, err, m);
  // every A tile is staged (the barrier inside tc_product) before any is overwritten
  if (ok && (row < 64 || two)) {
    float* out = (row < 64 ? a0 : a1) + (row & 63) * TILE + col0;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      reinterpret_cast<float4*>(out)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2],
                                                      v[4 * q + 3]);
  }
  tc_release(tmem);
}

// Trailing update A_ij -= L_ik L_jk^T for stored panel rows i >= j of column
// k: CTA (jj, p) updates the targets (jj + 2p, jj) and (jj + 2p + 1, jj).  The
// CTA whose first target is tile (k+1, k+1) then factors it (step k+1's
// potrf); the launch's last CTA does so when column k does not reach row k+1.
// grid = (max panel rows * pmax + 1, nmat), pmax = ceil(max panel rows / 2)
template <bool BF>
__global__ void __launch_bounds__(FB) k_syrk_tc(TileSetDev ts, int mat0, int nmat, int k, int pmax,
                                                float* __restrict__ tiles, ErrWord* err) {
  extern __shared__ __align__(1024) unsigned char dsm_tc[];
  if (grid_mat() >= nmat) return;
  const int m = mat0 + grid_mat();
  const int nt = ts.nt[m];
  if (k >= nt) return;
  const int fb = ts.vbase[m] / TILE;
  const int c0p = ts.colptr[fb + k];
  const int cnt = ts.colptr[fb + k + 1] - c0p;
  const long long tb = ts.tbase[m];
  if ((int)blockIdx.x == (int)gridDim.x - 1) {
    if (k + 1 < nt && ts.kmin[fb + k + 1] > k)
      potrf_tile<float>(tiles + tile_at(ts, tb, fb, k + 1, k + 1), dsm_tc, err, m,
                        tile_rows(ts, m, k + 1));
    return;
  }
  const int jj = (int)blockIdx.x / pmax, p = (int)blockIdx.x % pmax;
  const int ii0 = jj + 2 * p;
  if (jj >= cnt || ii0 >= cnt) return;
  const bool two = ii0 + 1 < cnt;
  const int j = ts.colidx[c0p + jj];
  const int i0 = ts.colidx[c0p + ii0];
  const float* l0 = tiles + tile_at(ts, tb, fb, i0, k);
  const float* l1 = two ? tiles + tile_at(ts, tb, fb, ts.colidx[c0p + ii0 + 1], k) : l0;
  const float* ljk = tiles + tile_at(ts, tb, fb, j, k);
  float* d0 = tiles + tile_at(ts, tb, fb, i0, j);
  float* d1 = two ? tiles + tile_at(ts, tb, fb, ts.colidx[c0p + ii0 + 1], j) : d0;
  float v[32];
  int row, col0;
  uint32_t tmem;
  const bool ok = tc_product<BF>(dsm_tc, l0, l1, ljk, v, row, col0, tmem, err, m);
  if (ok && (row < 64 || two)) {
    float* out = (row < 64 ? d0 : d1) + (row & 63) * TILE + col0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      float4 c = reinterpret_cast<float4*>(out)[q];
      c.x -= v[4 * q];
      c.y -= v[4 * q + 1];
      c.z -= v[4 * q + 2];
      c.w -= v[4 * q + 3];
      reinterpret_cast<float4*>(out)[q] = c;
    }
  }
  tc_release(tmem);
  if (ok && i0 == k + 1 && j == k + 1) {
    __threadfence();
    __syncthreads();  // the whole tile is written
    potrf_tile<float>(d0, dsm_tc, err, m, tile_rows(ts, m, k + 1));
  }
}

// ---------------------------------------------------------------------------
// FP64 panel and trailing update on the bf16 tensor cores by exact slicing
// (oz_tile.cuh): the same two-targets-per-CTA structure as the FP32 kernels,
// seven digit slices per operand, seven FP32 accumulator groups in 512 tensor-
// memory columns, one FP64 rounding per result.

__device__ __forceinline__ bool oz_product(unsigned char* dsm, const double* a0, const double* a1,
                                           const double* b, uint32_t& tmem, ErrWord* err, int m) {
  uint64_t* bar = reinterpret_cast<uint64_t*>(dsm + oz::BAR_OFF);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::smem_addr(tslot)),
                 "r"(oz::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    tc::mbar_init1(bar);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const int t = threadIdx.x;
  oz::stage_all(dsm, a0, a1, b);
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  tmem = *tslot;
  if (t == 0) {
    oz::issue_products(tmem, tc::smem_addr(dsm + oz::A_OFF), tc::smem_addr(dsm + oz::B_OFF));
    tc::mma_commit(bar);
  }
  const bool ok = tc::mbar_wait_bounded(bar, 0, 1ll << 24);
  tc::fence_after_sync();
  if (!ok && (t & 31) == 0 && atomicCAS(&err->code, 0, (int)SFCDD_ERR_TIMEOUT) == 0)
    err->index = m;
  return ok;
}

__device__ __forceinline__ void oz_release(uint32_t tmem) {
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(oz::TMEM_COLS)
                 : "memory");
}

// This thread's row (of the 128) and its 32 columns of D = A B^T, written to
// out0 (rows 0-63) or out1 (rows 64-127): overwritten (SUB = false) or
// subtracted from (SUB = true).
template <bool SUB>
__device__ __forceinline__ void oz_emit(const unsigned char* dsm, uint32_t tmem, double* out0,
                                        double* out1, bool two) {
  const int* ex = reinterpret_cast<const int*>(dsm + oz::E_OFF);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = 32 * (w & 3) + lane;
  const uint32_t tl = tmem + ((uint32_t)(32 * (w & 3)) << 16);
  const bool mine = row < 64 || two;
  double* out = (row < 64 ? out0 : out1) + (row & 63) * TILE;
#pragma unroll 1
  for (int q = 0; q < 4; ++q) {
    const int c0 = 32 * (w >> 2) + 8 * q;
    double v[8];
    oz::read_combine8(tl, c0, ex[row], ex + 128, v);  // every lane: .sync.aligned loads
    if (mine) {
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        double2* o = reinterpret_cast<double2*>(out + c0 + j);
        if (SUB) {
          double2 c = *o;
          c.x -= v[j];
          c.y -= v[j + 1];
          *o = c;
        } else {
          *o = make_double2(v[j], v[j + 1]);
        }
      }
    }
  }
}

// The FP64 tile-product kernels hold one CTA per SM (their shared memory and
// the whole TMEM), so they take the SM's register budget: __launch_bounds__
// with one block per SM keeps the fused diagonal factorization out of local
// memory.
// Panel L_ik = A_ik Linv_kk^T in FP64, two stored tiles of column k per CTA.
// grid = (ceil(max panel rows / 2), nmat)
__global__ void __launch_bounds__(FB, 1) k_trsm_oz(TileSetDev ts, int mat0, int nmat, int k,
                                                   double* __restrict__ tiles, ErrWord* err) {
  extern __shared__ __align__(1024) unsigned char dsm_oz[];
  if (grid_mat() >= nmat) return;
  const int m = mat0 + grid_mat();
  const int nt = ts.nt[m];
  if (k >= nt) return;
  const int fb = ts.vbase[m] / TILE;
  const int c0p = ts.colptr[fb + k];
  const int cnt = ts.colptr[fb + k + 1] - c0p;
  const int t0 = 2 * (int)blockIdx.x;
  if (t0 >= cnt) return;
  const bool two = t0 + 1 < cnt;
  const long long tb = ts.tbase[m];
  double* a0 = tiles + tile_at(ts, tb, fb, ts.colidx[c0p + t0], k);
  double* a1 = two ? tiles + tile_at(ts, tb, fb, ts.colidx[c0p + t0 + 1], k) : a0;
  const double* lkk = tiles + tile_at(ts, tb, fb, k, k);
  uint32_t tmem;
  // every A tile is staged (the barrier inside oz_product) before any is overwritten
  if (oz_product(dsm_oz, a0, a1, lkk, tmem, err, m)) oz_emit<false>(dsm_oz, tmem, a0, a1, two);
  oz_release(tmem);
}

// Trailing update A_ij -= L_ik L_jk^T in FP64; same target map as k_syrk_tc.
// grid = (max panel rows * pmax + 1, nmat), pmax = ceil(max panel rows / 2)
__global__ void __launch_bounds__(FB, 1) k_syrk_oz(TileSetDev ts, int mat0, int nmat, int k, int pmax,
                                                   double* __restrict__ tiles, ErrWord* err) {
  extern __shared__ __align__(1024) unsigned char dsm_oz[];
  if (grid_mat() >= nmat) return;
  const int m = mat0 + grid_mat();
  const int nt = ts.nt[m];
  if (k >= nt) return;
  const int fb = ts.vbase[m] / TILE;
  const int c0p = ts.colptr[fb + k];
  const int cnt = ts.colptr[fb + k + 1] - c0p;
  const long long tb = ts.tbase[m];
  if ((int)blockIdx.x == (int)gridDim.x - 1) {
    if (k + 1 < nt && ts.kmin[fb + k + 1] > k)
      potrf_tile<double>(tiles + tile_at(ts, tb, fb, k + 1, k + 1), dsm_oz, err, m,
                         tile_rows(ts, m, k + 1));
    return;
  }
  const int jj = (int)blockIdx.x / pmax, p = (int)blockIdx.x % pmax;
  const int ii0 = jj + 2 * p;
  if (jj >= cnt || ii0 >= cnt) return;
  const bool two = ii0 + 1 < cnt;
  const int j = ts.colidx[c0p + jj];
  const int i0 = ts.colidx[c0p + ii0];
  const double* l0 = tiles + tile_at(ts, tb, fb, i0, k);
  const double* l1 = two ? tiles + tile_at(ts, tb, fb, ts.colidx[c0p + ii0 + 1], k) : l0;
  const double* ljk = tiles + tile_at(ts, tb, fb, j, k);
  double* d0 = tiles + tile_at(ts, tb, fb, i0, j);
  double* d1 = two ? tiles + tile_at(ts, tb, fb, ts.colidx[c0p + ii0 + 1], j) : d0;
  uint32_t tmem;
  const bool ok = oz_product(dsm_oz, l0, l1, ljk, tmem, err, m);
  if (ok) oz_emit<true>(dsm_oz, tmem, d0, d1, two);
  oz_release(tmem);
  if (ok && i0 == k + 1 && j == k + 1) {
    __threadfence();
    __syncthreads();  // the whole tile is written
    potrf_tile<double>(d0, dsm_oz, err, m, tile_rows(ts, m, k + 1));
  }
}

// The FP64 factorization with its panel and trailing updates on the tensor cores.
static void factor_tiles_oz(const TileSetDev& ts, int mat0, int nmat, int max_nt,
                            const int* col_max, double* tiles, ErrWord* err, cudaStream_t s,
                            LaunchHook* hook) {
  const int sm_potrf = (2 * TILE + 1) * (TILE + 1) * (int)sizeof(double);
  const int sm_oz = (int)oz::SMEM_BYTES;
  cudaFuncSetAttribute(k_potrf<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_potrf);
  cudaFuncSetAttribute(k_trsm_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_oz);
  cudaFuncSetAttribute(k_syrk_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_oz);
  hook->before(SFCDD_K_POTRF);
  k_potrf<double><<<nmat, FB, sm_potrf, s>>>(ts, mat0, 0, tiles, err);
  hook->after(SFCDD_K_POTRF);
  for (int k = 0; k < max_nt; ++k) {
    const int rows = col_max[k];
    if (rows > 0) {
      const int pmax = (rows + 1) / 2;
      hook->before(SFCDD_K_TRSM);
      k_trsm_oz<<<mat_grid(pmax, nmat), FB, sm_oz, s>>>(ts, mat0, nmat, k, tiles, err);
      hook->after(SFCDD_K_TRSM);
      hook->before(SFCDD_K_SYRK);
      k_syrk_oz<<<mat_grid(rows * pmax + 1, nmat), FB, sm_oz, s>>>(ts, mat0, nmat, k, pmax, tiles,
                                                                    err);
      hook->after(SFCDD_K_SYRK);
    } else if (k + 1 < max_nt) {
      hook->before(SFCDD_K_POTRF);
      k_potrf<double><<<nmat, FB, sm_potrf, s>>>(ts, mat0, k + 1, tiles, err);
      hook->after(SFCDD_K_POTRF);
    }
  }
}

// The FP32 factorization with its panel and trailing updates on the tensor cores
// (BF: bf16 operands, the BF16 factorization; else the FP32-accurate TF32 split).
template <bool BF>
static void factor_tiles_tc(const TileSetDev& ts, int mat0, int nmat, int max_nt,
                            const int* col_max, float* tiles, ErrWord* err, cudaStream_t s,
                            LaunchHook* hook) {
  const int sm_potrf = (2 * TILE + 1) * (TILE + 1) * (int)sizeof(float);
  // the syrk launch's last CTA factors the next diagonal tile in the same shared memory
  const int sm_tc = std::max(tc_smem_bytes<BF>(), sm_potrf);
  cudaFuncSetAttribute(k_potrf<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_potrf);
  cudaFuncSetAttribute(k_trsm_tc<BF>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_tc);
  cudaFuncSetAttribute(k_syrk_tc<BF>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_tc);
  hook->before(SFCDD_K_POTRF);
  k_potrf<float><<<nmat, FB, sm_potrf, s>>>(ts, mat0, 0, tiles, err);
  hook->after(SFCDD_K_POTRF);
  for (int k = 0; k < max_nt; ++k) {
    const int rows = col_max[k];
    if (rows > 0) {
      const int pmax = (rows + 1) / 2;
      hook->before(SFCDD_K_TRSM);
      k_trsm_tc<BF><<<mat_grid(pmax, nmat), FB, sm_tc, s>>>(ts, mat0, nmat, k, tiles, err);
      hook->after(SFCDD_K_TRSM);
      hook->before(SFCDD_K_SYRK);
      k_syrk_tc<BF><<<mat_grid(rows * pmax + 1, nmat), FB, sm_tc, s>>>(ts, mat0, nmat, k, pmax,
                                                                        tiles, err);
      hook->after(SFCDD_K_SYRK);
    } else if (k + 1 < max_nt) {
      hook->before(SFCDD_K_POTRF);
      k_potrf<float><<<nmat, FB, sm_potrf, s>>>(ts, mat0, k + 1, tiles, err);
      hook->after(SFCDD_K_POTRF);
    }
  }
}

template <class T, int SPLIT>
static void factor_tiles_t(const TileSetDev& ts, int mat0, int nmat, int max_nt, const int* col_max,
                           T* tiles, int* diag_cnt, ErrWord* err, cudaStream_t s, LaunchHook* hook) {
  const int sm_potrf = (2 * TILE + 1) * (TILE + 1) * (int)sizeof(T);
  const int sm_gemm = std::max(2 * TILE * (TILE + 4), (2 * TILE + 1) * (TILE + 1)) * (int)sizeof(T);
  cudaFuncSetAttribute(k_potrf<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_potrf);
  cudaFuncSetAttribute(k_trsm<T, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_gemm);
  cudaFuncSetAttribute(k_syrk<T, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_gemm);
  // step k: panel (trsm), then trailing update fused with the factorization of
  // diagonal tile k+1; only step 0 and steps without a panel launch potrf alone
  hook->before(SFCDD_K_POTRF);
  k_potrf<T><<<nmat, FB, sm_potrf, s>>>(ts, mat0, 0, tiles, err);
  hook->after(SFCDD_K_POTRF);
  for (int k = 0; k < max_nt; ++k) {
    const int rows = col_max[k];
    if (rows > 0) {
      hook->before(SFCDD_K_TRSM);
      k_trsm<T, SPLIT><<<mat_grid(rows * SPLIT, nmat), FB, sm_gemm, s>>>(ts, mat0, nmat, k, tiles);
      hook->after(SFCDD_K_TRSM);
      hook->before(SFCDD_K_SYRK);
      k_syrk<T, SPLIT><<<mat_grid(rows * (rows + 1) / 2 * SPLIT + 1, nmat), FB, sm_gemm, s>>>(
          ts, mat0, nmat, k, tiles, diag_cnt, err);
      hook->after(SFCDD_K_SYRK);
    } else if (k + 1 < max_nt) {
      hook->before(SFCDD_K_POTRF);
      k_potrf<T><<<nmat, FB, sm_potrf, s>>>(ts, mat0, k + 1, tiles, err);
      hook->after(SFCDD_K_POTRF);
    }
  }
}

void factor_tiles(const TileSetDev& ts, int mat0, int nmat, int max_nt, const int* col_max,
                  void* tiles, Store st, int* diag_cnt, ErrWord* err, cudaStream_t s,
                  LaunchHook* hook, int split, bool tensor_cores, bool bf16_operands) {
  if (st == Store::F64 && tensor_cores) {
    factor_tiles_oz(ts, mat0, nmat, max_nt, col_max, (double*)tiles, err, s, hook);
  } else if (st == Store::F64) {
    if (split == 4)
      factor_tiles_t<double, 4>(ts, mat0, nmat, max_nt, col_max, (double*)tiles, diag_cnt, err, s,
                                hook);
    else
      factor_tiles_t<double, 1>(ts, mat0, nmat, max_nt, col_max, (double*)tiles, diag_cnt, err, s,
                                hook);
  } else if (tensor_cores && bf16_operands) {
    factor_tiles_tc<true>(ts, mat0, nmat, max_nt, col_max, (float*)tiles, err, s, hook);
  } else if (tensor_cores) {
    factor_tiles_tc<false>(ts, mat0, nmat, max_nt, col_max, (float*)tiles, err, s, hook);
  } else {
    factor_tiles_t<float, 1>(ts, mat0, nmat, max_nt, col_max, (float*)tiles, diag_cnt, err, s, hook);
  }
}

// A 64 x 64 row-major tile into a padded shared array, rows kept as rows.
template <class T>
__device__ __forceinline__ void load_plain(T (*dst)[TILE + 4], const T* __restrict__ src) {
  for (int e = threadIdx.x; e < TILE2; e += FB) dst[e / TILE][e % TILE] = src[e];
}

// acc[i][j] = sum_{s >= s0} Xt[s][r0 + i] Yt[s][c0 + j]
template <class T>
__device__ __forceinline__ void mma_4x4_from(T (&acc)[4][4], T (*Xt)[TILE + 4],
                                             T (*Yt)[TILE + 4], int r0, int c0, int s0,
                                             int s1 = TILE) {
#pragma unroll 4
  for (int s = s0; s < s1; ++s) {
    T xv[4], yv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      xv[i] = Xt[s][r0 + i];
      yv[i] = Yt[s][c0 + i];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) acc[i][jj] += xv[i] * yv[jj];
  }
}

// One stored tile per CTA.  With X = L_KK^{-1} (lower triangular, held in the
// diagonal slot): off-diagonal tile (I, K) -> Lh = L_IK X in place and Lh^T
// into ut; diagonal tile K -> E_K = X^T X into ut.  Both products only involve
// k >= column, so each warp starts its k loop at its first column (threads of
// a warp share a column block: c0 = 4 (tid / 16)).  grid = (max stored, nmat)
template <class T>
__global__ void __launch_bounds__(FB) k_unitize(TileSetDev ts, int mat0, int nmat,
                                                T* __restrict__ tiles,
                                                T* __restrict__ ut) {
  extern __shared__ __align__(16) unsigned char dsm_unit[];
  T (*Xt)[TILE + 4] = reinterpret_cast<T (*)[TILE + 4]>(dsm_unit);
  T (*Yt)[TILE + 4] = Xt + TILE;
  if (grid_mat() >= nmat) return;
  const int m = mat0 + grid_mat();
  const int nt = ts.nt[m];
  const int fb = ts.vbase[m] / TILE;
  if ((int)blockIdx.x >= stored_tiles(ts, fb, nt)) return;
  int I, K;
  skyline_decode(ts, fb, nt, blockIdx.x, I, K);
  const long long tb = ts.tbase[m];
  const T* xinv = tiles + tile_at(ts, tb, fb, K, K);
  T* tile = tiles + tile_at(ts, tb, fb, I, K);
  T* tout = ut + tile_at(ts, tb, fb, I, K);
  const int r0 = (threadIdx.x % 16) * 4, c0 = (threadIdx.x / 16) * 4;
  const int s0 = (threadIdx.x / 32) * 8;  // smallest column of the warp
  if (I == K) {
    load_plain<T>(Xt, xinv);  // Xt[s][a] = X[s][a]: E = X^T X
  } else {
    load_transposed<T>(Xt, tile);  // Xt[s][a] = L_IK[a][s]
    load_plain<T>(Yt, xinv);       // Yt[s][b] = X[s][b]: Lh = L_IK X
  }
  __syncthreads();
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  // a matrix's last tile row / column may hold fewer than TILE rows: the padding
  // is zero in L_IK and the identity in X_K, so only the inner index s < mK
  // contributes, and warps whose columns lie in the padding have nothing to do
  const int mK = tile_rows(ts, m, K);
  if (s0 < mK) mma_4x4_from<T>(acc, Xt, I == K ? Xt : Yt, r0, c0, s0, mK);
  if (I == K)  // E_K = X_K^T X_K is the identity on the padding
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (r0 + a == c0 + b && r0 + a >= mK) acc[a][b] = T(1);
  __syncthreads();
  // stage the result (rows in Xt) and its transpose (rows in Yt), then copy out
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      Xt[r0 + a][c0 + b] = acc[a][b];
      Yt[c0 + b][r0 + a] = acc[a][b];
    }
  __syncthreads();
  if (I == K) {
    for (int e = threadIdx.x; e < TILE2; e += FB) tout[e] = Xt[e / TILE][e % TILE];
  } else {
    for (int e = threadIdx.x; e < TILE2; e += FB) {
      tile[e] = Xt[e / TILE][e % TILE];
      tout[e] = Yt[e / TILE][e % TILE];
    }
  }
}

template <class T>
static void unitize_t(const TileSetDev& ts, int mat0, int nmat, int max_stored, T* tiles, T* ut,
                      cudaStream_t s) {
  if (nmat <= 0 || max_stored <= 0) return;
  const int sm = 2 * TILE * (TILE + 4) * (int)sizeof(T);
  cudaFuncSetAttribute(k_unitize<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  k_unitize<T><<<mat_grid(max_stored, nmat), FB, sm, s>>>(ts, mat0, nmat, tiles, ut);
}

// Zero rows of the off-block Lh tiles.  The Cholesky factor keeps the row
// envelope of A_i (no fill left of a row's first nonzero), and Lh = L D^{-1}
// keeps every zero row of L zero, so in tile row I the rows whose envelope
// starts inside the diagonal tile are zero in all of the row's off-block tiles.
// With the narrow local bands of curve-ordered subdomains that is most rows.
// The bound is taken from the stored values themselves (any nonzero bit
// pattern counts, -0 included), so skipping the rows beyond it is exact in every
// precision.  One warp per tile row, scanning each tile from its last row up.
template <int ES>
__global__ void k_offblock_rows(TileSetDev ts, int mat0, int nmat, const unsigned char* __restrict__ tiles,
                                int* __restrict__ nzr) {
  if (grid_mat() >= nmat) return;
  const int m = mat0 + grid_mat();
  const int I = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (I >= ts.nt[m]) return;  // whole warp
  const int fb = ts.vbase[m] / TILE;
  const long long tb = ts.tbase[m];
  constexpr int WPR = TILE * ES / 4;  // 32-bit words per tile row
  int last = 0;
  for (int K = ts.kmin[fb + I]; K < I; ++K) {
    const uint32_t* tp = reinterpret_cast<const uint32_t*>(tiles + tile_at(ts, tb, fb, I, K) * ES);
    for (int rr = TILE - 1; rr >= last; --rr) {
      uint32_t w = 0;
#pragma unroll
      for (int j = lane; j < WPR; j += 32) w |= __ldg(tp + rr * WPR + j);
      if (__any_sync(0xffffffffu, w != 0u)) {
        last = rr + 1;
        break;
      }
    }
  }
  if (lane == 0) nzr[fb + I] = last;
}

void launch_offblock_rows(const TileSetDev& ts, int mat0, int nmat, int max_nt, const void* tiles,
                          Store st, int* nzr, cudaStream_t s) {
  if (nmat <= 0 || max_nt <= 0) return;
  const dim3 grid = mat_grid((max_nt + 3) / 4, nmat);
  const unsigned char* t = static_cast<const unsigned char*>(tiles);
  switch (st) {
    case Store::F64: k_offblock_rows<8><<<grid, 128, 0, s>>>(ts, mat0, nmat, t, nzr); break;
    case Store::F32: k_offblock_rows<4><<<grid, 128, 0, s>>>(ts, mat0, nmat, t, nzr); break;
    default: k_offblock_rows<2><<<grid, 128, 0, s>>>(ts, mat0, nmat, t, nzr); break;
  }
}

// Packs the left halves of the FP64 transposed tiles whose source row bound is
// at most TILE / 2 (one CTA per stored tile; read all, then write in place).
__global__ void __launch_bounds__(FB) k_pack_half_tiles(TileSetDev ts, int mat0, int nmat,
                                                        double* __restrict__ ut,
                                                        const int* __restrict__ nzr) {
  __shared__ double half[TILE * (TILE / 2)];
  if (grid_mat() >= nmat) return;
  const int m = mat0 + grid_mat();
  const int nt = ts.nt[m];
  const int fb = ts.vbase[m] / TILE;
  if ((int)blockIdx.x >= stored_tiles(ts, fb, nt)) return;
  int I, K;
  skyline_decode(ts, fb, nt, blockIdx.x, I, K);
  if (I == K || nzr[fb + I] > TILE / 2) return;  // uniform over the CTA
  double* t = ut + tile_at(ts, ts.tbase[m], fb, I, K);
  for (int e = threadIdx.x; e < TILE * (TILE / 2); e += FB)
    half[e] = t[(e / (TILE / 2)) * TILE + e % (TILE / 2)];
  __syncthreads();
  for (int e = threadIdx.x; e < TILE * (TILE / 2); e += FB) t[e] = half[e];
}

void launch_pack_half_tiles(const TileSetDev& ts, int mat0, int nmat, int max_stored, double* ut,
                            const int* nzr, cudaStream_t s) {
  if (nmat <= 0 || max_stored <= 0) return;
  k_pack_half_tiles<<<mat_grid(max_stored, nmat), FB, 0, s>>>(ts, mat0, nmat, ut, nzr);
}

// ---------------------------------------------------------------------------
// Substitution form with cb-tile diagonal blocks (one matrix, FP64).  D_J is
// the lower block-triangular cb x cb-tile diagonal block J of the factor and
// X_J = D_J^{-1}; L = Lh blockdiag(D_J) with Lh_IK = sum_k L_{I,k} X_{k,K}
// over the tiles k of K's block (k >= K), and E_J = X_J^T X_J.  xs holds X_J
// as a cb x cb grid of tiles per block.

// acc += P Q on 64 x 64 tiles.  p_rowmajor: the tile at p holds P row-major
// (staged transposed, Xt[s][a] = P[a][s]); otherwise it holds P^T row-major
// (staged as is).  Q is row-major.
__device__ __forceinline__ void acc_product(double (&acc)[4][4], double (*Xt)[TILE + 4],
                                            double (*Yt)[TILE + 4], const double* __restrict__ p,
                                            bool p_rowmajor, const double* __restrict__ q,
                                            int r0, int c0) {
  __syncthreads();  // previous users of Xt / Yt are done
  if (p_rowmajor) load_transposed<double>(Xt, p);  // Xt[s][a] = P[a][s]
  else load_plain<double>(Xt, p);                  // p holds P^T: Xt[s][a] = P^T[s][a] = P[a][s]
  load_plain<double>(Yt, q);                       // Yt[s][b] = Q[s][b]
  __syncthreads();
  mma_4x4_from<double>(acc, Xt, Yt, r0, c0, 0);
}

__device__ __forceinline__ long long xs_off(int cb, int J, int i, int j) {
  return ((long long)(J * cb + i) * cb + j) * TILE2;
}

// Diagonal d of every block: X_{j+d, j} = -X_{j+d,j+d} sum_{k=j}^{j+d-1} L_{j+d,k} X_{k,j}
// (d = 0 copies the stored inverses).  grid = (cb, number of blocks)
__global__ void __launch_bounds__(FB) k_sb_inverse(TileSetDev ts, int cb, int d,
                                                   const double* __restrict__ tiles,
                                                   double* __restrict__ xs) {
  extern __shared__ __align__(16) unsigned char dsm_sbi[];
  double (*Xt)[TILE + 4] = reinterpret_cast<double (*)[TILE + 4]>(dsm_sbi);
  double (*Yt)[TILE + 4] = Xt + TILE;
  const int J = blockIdx.y, j = blockIdx.x, i = j + d;
  const int nt = ts.nt[0];
  const int blk0 = J * cb;
  const int nb = min(cb, nt - blk0);
  if (i >= nb) return;
  const int fb = ts.vbase[0] / TILE;
  const long long tb = ts.tbase[0];
  double* out = xs + xs_off(cb, J, i, j);
  if (d == 0) {
    const double* src = tiles + tile_at(ts, tb, fb, blk0 + i, blk0 + i);
    for (int e = threadIdx.x; e < TILE2; e += FB) out[e] = src[e];
    return;
  }
  const int r0 = (threadIdx.x % 16) * 4, c0 = (threadIdx.x / 16) * 4;
  double acc[4][4] = {};
  for (int k = j; k < i; ++k)
    acc_product(acc, Xt, Yt, tiles + tile_at(ts, tb, fb, blk0 + i, blk0 + k), true,
                xs + xs_off(cb, J, k, j), r0, c0);
  // S -> Yt, then X_ij = -X_ii S
  __syncthreads();
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) Yt[r0 + a][c0 + b] = acc[a][b];
  load_transposed<double>(Xt, xs + xs_off(cb, J, i, i));
  __syncthreads();
  double x[4][4] = {};
  mma_4x4_from<double>(x, Xt, Yt, r0, c0, 0);
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) out[(r0 + a) * TILE + c0 + b] = -x[a][b];
}

// One stored tile (I, K) per CTA.  Inside a block (I, K in block J, a >= b
// their offsets): E_ab = sum_{k >= a} X_ka^T X_kb into ut, and E_ba = E_ab^T
// into the tiles slot when a > b.  Below the block: Lh_IK^T into ut (the
// tiles slot still holds L and is read by the other tiles of row I).
__global__ void __launch_bounds__(FB) k_sb_unitize(TileSetDev ts, int cb, double* __restrict__ tiles,
                                                   double* __restrict__ ut,
                                                   const double* __restrict__ xs) {
  extern __shared__ __align__(16) unsigned char dsm_sbu[];
  double (*Xt)[TILE + 4] = reinterpret_cast<double (*)[TILE + 4]>(dsm_sbu);
  double (*Yt)[TILE + 4] = Xt + TILE;
  const int nt = ts.nt[0];
  const int fb = ts.vbase[0] / TILE;
  if ((int)blockIdx.x >= stored_tiles(ts, fb, nt)) return;
  int I, K;
  skyline_decode(ts, fb, nt, blockIdx.x, I, K);
  const long long tb = ts.tbase[0];
  const int J = K / cb, blk0 = J * cb;
  const int nb = min(cb, nt - blk0);
  const int b = K - blk0;
  const int r0 = (threadIdx.x % 16) * 4, c0 = (threadIdx.x / 16) * 4;
  double acc[4][4] = {};
  const bool inside = I < blk0 + nb;
  if (inside) {
    const int aa = I - blk0;
    // X_ka^T X_kb: Xt[s][p] = X_ka[s][p] (plain = P^T given), Yt = X_kb
    for (int k = aa; k < nb; ++k)
      acc_product(acc, Xt, Yt, xs + xs_off(cb, J, k, aa), false,
                  xs + xs_off(cb, J, k, b), r0, c0);
  } else {
    for (int k = b; k < nb; ++k)
      acc_product(acc, Xt, Yt, tiles + tile_at(ts, tb, fb, I, blk0 + k), true,
                  xs + xs_off(cb, J, k, b), r0, c0);
  }
  __syncthreads();
  for (int a = 0; a < 4; ++a)
    for (int q = 0; q < 4; ++q) {
      Xt[r0 + a][c0 + q] = acc[a][q];
      Yt[c0 + q][r0 + a] = acc[a][q];
    }
  __syncthreads();
  double* uo = ut + tile_at(ts, tb, fb, I, K);
  if (inside) {
    for (int e = threadIdx.x; e < TILE2; e += FB) uo[e] = Xt[e / TILE][e % TILE];
    if (I > K) {
      double* lo = tiles + tile_at(ts, tb, fb, I, K);
      for (int e = threadIdx.x; e < TILE2; e += FB) lo[e] = Yt[e / TILE][e % TILE];
    }
  } else {
    for (int e = threadIdx.x; e < TILE2; e += FB) uo[e] = Yt[e / TILE][e % TILE];
  }
}

// Below-block tiles: tiles(I, K) = ut(I, K)^T = Lh_IK.
__global__ void __launch_bounds__(FB) k_sb_transpose(TileSetDev ts, int cb, double* __restrict__ tiles,
                                                     const double* __restrict__ ut) {
  __shared__ double t[TILE][TILE + 1];
  const int nt = ts.nt[0];
  const int fb = ts.vbase[0] / TILE;
  if ((int)blockIdx.x >= stored_tiles(ts, fb, nt)) return;
  int I, K;
  skyline_decode(ts, fb, nt, blockIdx.x, I, K);
  const int blk0 = K / cb * cb;
  if (I < min(blk0 + cb, nt)) return;
  const long long off = tile_at(ts, ts.tbase[0], fb, I, K);
  for (int e = threadIdx.x; e < TILE2; e += FB) t[e / TILE][e % TILE] = ut[off + e];
  __syncthreads();
  for (int e = threadIdx.x; e < TILE2; e += FB) tiles[off + e] = t[e % TILE][e / TILE];
}

void unitize_blocks(const TileSetDev& ts, int nt, int cb, int stored, double* tiles, double* ut,
                    double* xs, cudaStream_t s) {
  const int sm = 2 * TILE * (TILE + 4) * (int)sizeof(double);
  cudaFuncSetAttribute(k_sb_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_sb_unitize, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  const int nblk = (nt + cb - 1) / cb;
  for (int d = 0; d < cb; ++d) k_sb_inverse<<<dim3(cb - d, nblk), FB, sm, s>>>(ts, cb, d, tiles, xs);
  k_sb_unitize<<<stored, FB, sm, s>>>(ts, cb, tiles, ut, xs);
  k_sb_transpose<<<stored, FB, 0, s>>>(ts, cb, tiles, ut);
}

void unitize_tiles(const TileSetDev& ts, int mat0, int nmat, int max_stored, void* tiles, void* ut,
                   Store st, cudaStream_t s) {
  if (st == Store::F64)
    unitize_t<double>(ts, mat0, nmat, max_stored, (double*)tiles, (double*)ut, s);
  else
    unitize_t<float>(ts, mat0, nmat, max_stored, (float*)tiles, (float*)ut, s);
}

__global__ void k_convert_f32_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out,
                                   long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = __float2bfloat16_rn(in[i]);
}

void launch_convert_f32_bf16(const float* in, __nv_bfloat16* out, long long n, cudaStream_t s) {
  k_convert_f32_bf16<<<152 * 16, 256, 0, s>>>(in, out, n);
}

// Dense symmetric N x N copy (row-major) of an FP64 tile-skyline matrix before
// factorization (introspection only), rows and columns in ascending cyclic
// curve order (mapped through the local numbering); entries outside the
// envelope are zero.
__global__ void k_unpack_dense(TileSetDev ts, int m, const double* __restrict__ tiles,
                               double* __restrict__ dense, const int* __restrict__ rowmap) {
  const int n = ts.n[m];
  const int fb = ts.vbase[m] / TILE;
  const int* linv = rowmap ? rowmap : (ts.linv ? ts.linv + ts.vbase[m] : nullptr);
  const long long tot = (long long)n * n;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += stride) {
    int r = (int)(e / n), c = (int)(e % n);
    if (linv) {
      r = linv[r];
      c = linv[c];
    }
    if (c > r) {
      const int t = r;
      r = c;
      c = t;
    }
    const int a = r / TILE, b = c / TILE;
    double v = 0.0;
    if (b >= ts.kmin[fb + a])
      v = tiles[tile_at(ts, ts.tbase[m], fb, a, b) + (r % TILE) * TILE + (c % TILE)];
    dense[e] = v;
  }
}

__global__ void k_lorder_keys(TileSetDev ts, const int* __restrict__ mstart, const int* __restrict__ mN,
                              const int* __restrict__ mcbase, const int* __restrict__ lbase,
                              const unsigned* __restrict__ code, unsigned long long* __restrict__ keys,
                              unsigned* __restrict__ vals, int nmat) {
  const int m = grid_mat();
  if (m >= nmat) return;
  const int n = ts.n[m], start = mstart[m], N = mN[m];
  const unsigned* cs = code + mcbase[m];
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n; o += gridDim.x * blockDim.x) {
    int p = start + o;
    if (p >= N) p -= N;
    keys[lbase[m] + o] = ((unsigned long long)m << 32) | cs[p];
    vals[lbase[m] + o] = (unsigned)o;
  }
}

__global__ void k_lorder_scatter(TileSetDev ts, const int* __restrict__ mstart, const int* __restrict__ mN,
                                 const int* __restrict__ lbase, long long total,
                                 const unsigned long long* __restrict__ keys,
                                 const unsigned* __restrict__ vals, int* __restrict__ lperm,
                                 int* __restrict__ linv) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += stride) {
    const int m = (int)(keys[k] >> 32);
    const int r = (int)(k - lbase[m]);
    const int o = (int)vals[k];
    int p = mstart[m] + o;
    if (p >= mN[m]) p -= mN[m];
    const int vb = ts.vbase[m];
    lperm[vb + r] = p;
    linv[vb + o] = r;
  }
}

void local_order_lex(const TileSetDev& ts, int nmat, int max_n, const int* mstart, const int* mN,
                     const int* mcbase, const int* lbase, long long total, const unsigned* code,
                     unsigned long long* keys, unsigned* vals, void* temp, int* lperm, int* linv,
                     cudaStream_t s) {
  int mbits = 1;
  while ((1 << mbits) < nmat) ++mbits;
  k_lorder_keys<<<mat_grid((max_n + 255) / 256, nmat), 256, 0, s>>>(ts, mstart, mN, mcbase, lbase,
                                                                     code, keys, vals, nmat);
  radix_sort_pairs(keys, vals, (int)total, 32 + mbits, temp, s, nullptr);
  k_lorder_scatter<<<152 * 8, 256, 0, s>>>(ts, mstart, mN, lbase, total, keys, vals, lperm, linv);
}

void launch_unpack_dense(const TileSetDev& ts, int m, const double* tiles, double* dense,
                         const int* rowmap, cudaStream_t s) {
  k_unpack_dense<<<152 * 8, 256, 0, s>>>(ts, m, tiles, dense, rowmap);
}

// ---------------------------------------------------------------------------
// Coarse-block adjacency (input of the coarse numbering): one warp per coarse
// block b walks the block's points and their 2d neighbours, 32 candidates at a
// time.  A candidate is kept if it is another block, not yet in b's list and
// the lowest lane holding that block in its chunk (warp match), so each list
// ends up with every adjacent block exactly once, in order of first sight.
constexpr int ADJ_WARPS = 4;

__global__ void __launch_bounds__(ADJ_WARPS * 32)
    k_coarse_adjacency(GridDev g, PartDev pd, const unsigned* __restrict__ code,
                       const int* __restrict__ invpad, int maxdeg, int* __restrict__ adj,
                       int* __restrict__ deg) {
  extern __shared__ int sm_adj[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = blockIdx.x * ADJ_WARPS + w;
  const int N0 = pd.q * pd.P;
  if (b >= N0) return;  // whole warp
  int* list = sm_adj + w * maxdeg;
  int bstart, bsize;
  coarse_block_range(pd, b, bstart, bsize);
  const int nd = 2 * g.d;
  const int ncand = bsize * nd;
  int cnt = 0;
  bool overflow = false;
  for (int c0 = 0; c0 < ncand; c0 += 32) {
    const int k = c0 + lane;
    int nb = -1;
    if (k < ncand) {
      const int u = k / nd, dir = k % nd;
      const int q = neighbour(g, invpad, code[bstart + u], dir >> 1, dir & 1);
      if (q >= 0) nb = coarse_block_of(pd, q);
    }
    bool keep = nb >= 0 && nb != b;
    const int listed = cnt < maxdeg ? cnt : maxdeg;
    for (int i = 0; keep && i < listed; ++i)
      if (list[i] == nb) keep = false;
    // lanes with equal candidates: only the lowest keeps it (others get distinct keys)
    const unsigned same = __match_any_sync(0xffffffffu, keep ? nb : -2 - lane);
    if (keep && (__ffs(same) - 1) != lane) keep = false;
    const unsigned kb = __ballot_sync(0xffffffffu, keep);
    const int pos = cnt + __popc(kb & ((1u << lane) - 1u));
    if (keep) {
      if (pos < maxdeg) list[pos] = nb;
      else overflow = true;
    }
    cnt += __popc(kb);
    __syncwarp();
  }
  overflow = __any_sync(0xffffffffu, overflow) || cnt > maxdeg;
  for (int i = lane; i < cnt && !overflow; i += 32) adj[(long long)b * maxdeg + i] = list[i];
  if (lane == 0) deg[b] = overflow ? -1 : cnt;
}

void launch_coarse_adjacency(const GridDev& g, const PartDev& pd, const unsigned* code,
                             const int* invpad, int maxdeg, int* adj, int* deg, cudaStream_t s) {
  const int N0 = pd.q * pd.P;
  const int smem = ADJ_WARPS * maxdeg * (int)sizeof(int);
  cudaFuncSetAttribute(k_coarse_adjacency, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_coarse_adjacency<<<(N0 + ADJ_WARPS - 1) / ADJ_WARPS, ADJ_WARPS * 32, smem, s>>>(
      g, pd, code, invpad, maxdeg, adj, deg);
}

}  // namespace sfcdd
