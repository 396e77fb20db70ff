// Device building blocks shared by the single-problem and the batched kernels.
// Positions, codes and invpad tables are those of ONE problem (a batch passes
// pointers offset to its subgrid).
#pragma once
#include "sfcdd_internal.cuh"

namespace sfcdd {

// packed lower-triangular index -> (a, b), a >= b
__device__ __forceinline__ void tri_decode(int idx, int& a, int& b) {
  int t = (int)((sqrt(8.0 * idx + 1.0) - 1.0) * 0.5);
  while ((t + 1) * (t + 2) / 2 <= idx) ++t;
  while (t * (t + 1) / 2 > idx) --t;
  a = t;
  b = idx - t * (t + 1) / 2;
}

// stored tile number t of the matrix whose tile rows start at fb -> (I, K)
__device__ __forceinline__ void skyline_decode(const TileSetDev& ts, int fb, int nt, int t, int& I,
                                               int& K) {
  int lo = 0, hi = nt - 1;
  while (lo < hi) {  // last I with rowoff[I] <= t
    const int mid = (lo + hi + 1) >> 1;
    if (ts.rowoff[fb + mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  I = lo;
  K = ts.kmin[fb + I] + (t - ts.rowoff[fb + I]);
}

__device__ __forceinline__ int stored_tiles(const TileSetDev& ts, int fb, int nt) {
  return ts.rowoff[fb + nt - 1] + (nt - ts.kmin[fb + nt - 1]);
}

// Axis-j neighbour (s = 0: minus, 1: plus) of the point with code c: its curve
// position, or -1 at the Dirichlet boundary.
__device__ __forceinline__ int neighbour(const GridDev& g, const int* __restrict__ invpad,
                                         unsigned c, int j, int s) {
  const unsigned kj = (c >> g.off[j]) & ((1u << g.lev[j]) - 1u);
  const unsigned unit = 1u << g.off[j];
  if (s == 0) return kj > 1u ? __ldg(&invpad[c - unit]) : -1;
  return kj < (unsigned)g.size[j] ? __ldg(&invpad[c + unit]) : -1;
}

// Local numbering of a subdomain (start, n): local row r sits at curve position
// lperm[r] (lperm null: start + r, cyclic), and the point at offset
// o = (p - start) mod N inside the range has local row linv[o] (null: o).
struct LocalOrder {
  const int* lperm;
  const int* linv;
  __device__ __forceinline__ int pos(const GridDev& g, int start, int r) const {
    if (lperm) return lperm[r];
    int p = start + r;
    return p >= g.N ? p - g.N : p;
  }
  // local row of curve position q, or -1 if q lies outside the range
  __device__ __forceinline__ int row(const GridDev& g, int start, int n, int q) const {
    int o = q - start;
    if (o < 0) o += g.N;
    if (o >= n) return -1;
    return linv ? linv[o] : o;
  }
};

// Smallest local column with a nonzero in row r of the local matrix that starts
// at curve position `start` and has n rows (Cholesky envelope of the row).
__device__ __forceinline__ int envelope_row(const GridDev& g, const unsigned* __restrict__ code,
                                            const int* __restrict__ invpad, int start, int n,
                                            LocalOrder lo, int r) {
  const unsigned c = code[lo.pos(g, start, r)];
  int first = r;
  for (int j = 0; j < g.d; ++j)
    for (int s = 0; s < 2; ++s) {
      const int q = neighbour(g, invpad, c, j, s);
      if (q < 0) continue;
      const int cg = lo.row(g, start, n, q);
      if (cg >= 0 && cg < first) first = cg;
    }
  return first;
}

// Smallest coarse row adjacent to the row of the block of curve position p
// (returned in a).
__device__ __forceinline__ int envelope_coarse_point(const GridDev& g, const PartDev& pd,
                                                     const unsigned* __restrict__ code,
                                                     const int* __restrict__ invpad, int p,
                                                     int& a) {
  a = coarse_row(pd, coarse_block_of(pd, p));
  const unsigned c = code[p];
  int first = a;
  for (int j = 0; j < g.d; ++j)
    for (int s = 0; s < 2; ++s) {
      const int q = neighbour(g, invpad, c, j, s);
      if (q >= 0) first = min(first, coarse_row(pd, coarse_block_of(pd, q)));
    }
  return first;
}

// Tile (a, b) of the local matrix (start, n) into shared memory sm (TILE^2
// doubles, zeroed by the caller); threads 0..TILE-1 each fill one row.
__device__ __forceinline__ void assemble_local_tile(const GridDev& g,
                                                    const unsigned* __restrict__ code,
                                                    const int* __restrict__ invpad, int start,
                                                    int n, LocalOrder lo, int a, int b,
                                                    double* sm) {
  if (threadIdx.x >= TILE) return;
  const int tr = threadIdx.x;
  const int rg = a * TILE + tr;
  if (rg >= n) {
    if (a == b) sm[tr * TILE + tr] = 1.0;  // padding: identity
    return;
  }
  if (a == b) sm[tr * TILE + tr] = g.diag;
  const unsigned c = code[lo.pos(g, start, rg)];
  for (int j = 0; j < g.d; ++j)
    for (int s = 0; s < 2; ++s) {
      const int q = neighbour(g, invpad, c, j, s);
      if (q < 0) continue;
      const int cg = lo.row(g, start, n, q);
      if (cg >= 0 && cg < rg && cg >= b * TILE && cg < (b + 1) * TILE)
        sm[tr * TILE + (cg - b * TILE)] = -g.w[j];
    }
}

// Tile (R, C) of the coarse matrix A_0 = R_0 A R_0^T (eq. csm), rows and
// columns in the coarse factor's numbering, into acc (TILE^2 doubles) using cnt
// (TILE^2 ints) for the integer edge counts of each axis; 4 threads per coarse
// row walk the points of the row's block.  Needs FB >= 256.
__device__ __forceinline__ void assemble_coarse_tile(const GridDev& g, const PartDev& pd, int N0,
                                                     const unsigned* __restrict__ code,
                                                     const int* __restrict__ invpad, int R, int C,
                                                     double* acc, int* cnt) {
  const int nthr = blockDim.x;
  const int tr = threadIdx.x >> 2, sub = threadIdx.x & 3;
  const int arow = R * TILE + tr;
  int bstart = 0, bsize = 0;
  if (threadIdx.x < 4 * TILE && arow < N0)
    coarse_block_range(pd, coarse_block_at(pd, arow), bstart, bsize);
  for (int k = threadIdx.x; k < TILE2; k += nthr) {
    const int r = k / TILE, c = k % TILE;
    const int ar = R * TILE + r, bc = C * TILE + c;
    double v = 0.0;
    if (ar == bc) {
      if (ar < N0) {
        int bs, bn;
        coarse_block_range(pd, coarse_block_at(pd, ar), bs, bn);
        v = (double)bn * g.diag;
      } else {
        v = 1.0;  // padding: identity
      }
    }
    acc[k] = v;
  }
  for (int j = 0; j < g.d; ++j) {
    for (int k = threadIdx.x; k < TILE2; k += nthr) cnt[k] = 0;
    __syncthreads();
    if (threadIdx.x < 4 * TILE && arow < N0) {
      for (int u = sub; u < bsize; u += 4) {
        const unsigned c = code[bstart + u];
        for (int s = 0; s < 2; ++s) {
          const int q = neighbour(g, invpad, c, j, s);
          if (q < 0) continue;
          const int bcol = coarse_row(pd, coarse_block_of(pd, q));
          if (bcol >= C * TILE && bcol < (C + 1) * TILE && bcol <= arow)
            atomicAdd(&cnt[tr * TILE + (bcol - C * TILE)], 1);
        }
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < TILE2; k += nthr)
      if (cnt[k]) acc[k] -= g.w[j] * (double)cnt[k];
    __syncthreads();
  }
}

// (A x)_p for the matrix-free stencil in curve order.
template <int D>
__device__ __forceinline__ double stencil_point(const GridDev& g, const unsigned* __restrict__ code,
                                                const int* __restrict__ invpad,
                                                const double* __restrict__ x, int p, double& xp) {
  const unsigned c = __ldg(&code[p]);
  xp = __ldg(&x[p]);
  double v = g.diag * xp;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const unsigned kj = (c >> g.off[j]) & ((1u << g.lev[j]) - 1u);
    const unsigned unit = 1u << g.off[j];
    if (kj > 1u) v -= g.w[j] * __ldg(&x[__ldg(&invpad[c - unit])]);
    if (kj < (unsigned)g.size[j]) v -= g.w[j] * __ldg(&x[__ldg(&invpad[c + unit])]);
  }
  return v;
}

// z_p = d_0[block(p)] + sum_i omega_i d_i[row_i(p)] (eq. addSW), reading the
// coarse result at dvec[coarse_base + coarse_row(block)] and subdomain i's result at
// dvec[lvbase(i) + row], row = linv[lvbase(i) + offset] (linv null: the offset);
// mode 0 two-level, 1 one level, 2 coarse only.
template <class LocalBase>
__device__ __forceinline__ double prolong_point(const PartDev& pd, int mode,
                                                const double* __restrict__ dvec, int coarse_base,
                                                LocalBase lvbase, const int* __restrict__ linv,
                                                int p) {
  double v = 0.0;
  if (mode != 1) v = __ldg(&dvec[coarse_base + coarse_row(pd, coarse_block_of(pd, p))]);
  if (mode != 2) {
    const int ncand = min(2 * pd.g + 3, pd.P);
    const int t = tilde_of(pd, p);
    int i = t - pd.g - 1;
    i = ((i % pd.P) + pd.P) % pd.P;
    for (int k = 0; k < ncand; ++k) {
      int o = p - __ldg(&pd.start[i]);
      if (o < 0) o += pd.N;
      if (o < __ldg(&pd.len[i])) {
        const int vb = lvbase(i);
        const int row = linv ? __ldg(&linv[vb + o]) : o;
        v += __ldg(&pd.omega[i]) * __ldg(&dvec[vb + row]);
      }
      if (++i == pd.P) i = 0;
    }
  }
  return v;
}

}  // namespace sfcdd
