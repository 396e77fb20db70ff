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
// matrices: per step k one launch factors the diagonal tiles (and inverts the
// factor's diagonal block in place), one solves the panel, one updates the
// trailing lower triangle.
#include "sfcdd_internal.cuh"

namespace sfcdd {

constexpr int FB = 256;

// packed lower-triangular tile index -> (a, b)
__device__ __forceinline__ void tri_decode(int idx, int& a, int& b) {
  int t = (int)((sqrt(8.0 * idx + 1.0) - 1.0) * 0.5);
  while ((t + 1) * (t + 2) / 2 <= idx) ++t;
  while (t * (t + 1) / 2 > idx) --t;
  a = t;
  b = idx - t * (t + 1) / 2;
}

template <class T>
__device__ __forceinline__ T from_double(double v) { return T(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_double<__nv_bfloat16>(double v) {
  return __float2bfloat16_rn((float)v);
}

// ---------------------------------------------------------------------------
// Local matrices.  grid = (max tiles per matrix, nmat); one CTA per tile.
template <class T>
__global__ void __launch_bounds__(FB) k_assemble_local(GridDev g, PartDev pd,
                                                       const unsigned* __restrict__ code,
                                                       const int* __restrict__ invpad,
                                                       TileSetDev ts, int mat0, T* __restrict__ tiles) {
  __shared__ double sm[TILE2];
  const int m = mat0 + blockIdx.y;
  const int nt = ts.nt[m];
  const int idx = blockIdx.x;
  if (idx >= nt * (nt + 1) / 2) return;
  int a, b;
  tri_decode(idx, a, b);
  for (int k = threadIdx.x; k < TILE2; k += FB) sm[k] = 0.0;
  __syncthreads();
  const int n = ts.n[m];
  const int start = pd.start[m];
  if (threadIdx.x < TILE) {
    const int tr = threadIdx.x;
    const int rg = a * TILE + tr;
    if (rg >= n) {
      if (a == b) sm[tr * TILE + tr] = 1.0;  // padding: identity
    } else {
      int p = start + rg;
      if (p >= g.N) p -= g.N;
      if (a == b) sm[tr * TILE + tr] = g.diag;
      const unsigned c = code[p];
      for (int j = 0; j < g.d; ++j) {
        const unsigned kj = (c >> g.off[j]) & ((1u << g.lev[j]) - 1u);
        const unsigned unit = 1u << g.off[j];
        for (int s = 0; s < 2; ++s) {
          if (s == 0 && kj <= 1u) continue;
          if (s == 1 && kj >= (unsigned)g.size[j]) continue;
          const int q = invpad[s == 0 ? c - unit : c + unit];
          int cg = q - start;
          if (cg < 0) cg += g.N;
          if (cg < n && cg < rg && cg >= b * TILE && cg < (b + 1) * TILE)
            sm[tr * TILE + (cg - b * TILE)] = -g.w[j];
        }
      }
    }
  }
  __syncthreads();
  T* out = tiles + ts.tbase[m] + (long long)idx * TILE2;
  for (int k = threadIdx.x; k < TILE2; k += FB) out[k] = from_double<T>(sm[k]);
}

void launch_assemble_local(const GridDev& g, const PartDev& pd, const unsigned* code,
                           const int* invpad, const TileSetDev& ts, int mat0, int nmat, int max_tiles,
                           void* tiles, Store st, cudaStream_t s) {
  dim3 grid(max_tiles, nmat);
  switch (st) {
    case Store::F64:
      k_assemble_local<double><<<grid, FB, 0, s>>>(g, pd, code, invpad, ts, mat0, (double*)tiles);
      break;
    case Store::F32:
      k_assemble_local<float><<<grid, FB, 0, s>>>(g, pd, code, invpad, ts, mat0, (float*)tiles);
      break;
    default:
      k_assemble_local<__nv_bfloat16><<<grid, FB, 0, s>>>(g, pd, code, invpad, ts, mat0,
                                                          (__nv_bfloat16*)tiles);
      break;
  }
}

// ---------------------------------------------------------------------------
// Coarse matrix tiles (single matrix, nt0 tile rows).  One CTA per lower tile;
// 4 threads per coarse row walk the points of the row's block.
__global__ void __launch_bounds__(FB) k_assemble_coarse(GridDev g, PartDev pd,
                                                        const unsigned* __restrict__ code,
                                                        const int* __restrict__ invpad, int N0,
                                                        double* __restrict__ tiles) {
  extern __shared__ __align__(16) unsigned char dsm_coarse[];
  double* acc = reinterpret_cast<double*>(dsm_coarse);
  int* cnt = reinterpret_cast<int*>(acc + TILE2);
  int R, C;
  tri_decode(blockIdx.x, R, C);
  const int tr = threadIdx.x >> 2, sub = threadIdx.x & 3;
  const int arow = R * TILE + tr;
  // block of coarse row arow
  int bstart = 0, bsize = 0;
  if (arow < N0) {
    const int t = arow / pd.q, mm = arow % pd.q;
    const int n = tilde_size(pd, t);
    const int bf = n / pd.q, br = n % pd.q;
    bstart = tilde_off(pd, t) + (mm < br ? mm * (bf + 1) : br * (bf + 1) + (mm - br) * bf);
    bsize = mm < br ? bf + 1 : bf;
  }
  for (int k = threadIdx.x; k < TILE2; k += FB) {
    const int r = k / TILE, c = k % TILE;
    const int ar = R * TILE + r, bc = C * TILE + c;
    double v = 0.0;
    if (ar == bc) {
      if (ar < N0) {
        const int t = ar / pd.q, mm = ar % pd.q;
        const int n = tilde_size(pd, t);
        const int bf = n / pd.q, br = n % pd.q;
        v = (double)(mm < br ? bf + 1 : bf) * g.diag;
      } else {
        v = 1.0;  // padding: identity
      }
    }
    acc[k] = v;
  }
  for (int j = 0; j < g.d; ++j) {
    for (int k = threadIdx.x; k < TILE2; k += FB) cnt[k] = 0;
    __syncthreads();
    if (arow < N0) {
      const unsigned unit = 1u << g.off[j];
      for (int u = sub; u < bsize; u += 4) {
        const unsigned c = code[bstart + u];
        const unsigned kj = (c >> g.off[j]) & ((1u << g.lev[j]) - 1u);
        for (int s = 0; s < 2; ++s) {
          if (s == 0 && kj <= 1u) continue;
          if (s == 1 && kj >= (unsigned)g.size[j]) continue;
          const int q = invpad[s == 0 ? c - unit : c + unit];
          const int bcol = coarse_block_of(pd, q);
          if (bcol >= C * TILE && bcol < (C + 1) * TILE && bcol <= arow)
            atomicAdd(&cnt[tr * TILE + (bcol - C * TILE)], 1);
        }
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < TILE2; k += FB)
      if (cnt[k]) acc[k] -= g.w[j] * (double)cnt[k];
    __syncthreads();
  }
  double* out = tiles + (long long)blockIdx.x * TILE2;
  for (int k = threadIdx.x; k < TILE2; k += FB) out[k] = acc[k];
}

void launch_assemble_coarse(const GridDev& g, const PartDev& pd, const unsigned* code,
                            const int* invpad, int N0, int nt0, double* tiles, double* dense,
                            cudaStream_t s) {
  (void)dense;
  const int ntiles = nt0 * (nt0 + 1) / 2;
  const int smem = TILE2 * (int)(sizeof(double) + sizeof(int));
  cudaFuncSetAttribute(k_assemble_coarse, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_assemble_coarse<<<ntiles, FB, smem, s>>>(g, pd, code, invpad, N0, tiles);
}

// ---------------------------------------------------------------------------
// Factorization kernels, compute type T (double or float), storage T.

// Diagonal tile k of every matrix with nt > k: Cholesky in shared memory, then
// the inverse of the lower-triangular factor block replaces the tile.
template <class T>
__global__ void __launch_bounds__(FB) k_potrf(TileSetDev ts, int mat0, int k, T* __restrict__ tiles,
                                              ErrWord* err) {
  extern __shared__ __align__(16) unsigned char dsm_potrf[];
  T (*L)[TILE + 1] = reinterpret_cast<T (*)[TILE + 1]>(dsm_potrf);
  T (*X)[TILE + 1] = L + TILE;
  T& s_inv = X[TILE][0];
  const int m = mat0 + blockIdx.x;
  if (ts.nt[m] <= k) return;
  T* tp = tiles + ts.tbase[m] + (long long)(k * (k + 1) / 2 + k) * TILE2;
  for (int e = threadIdx.x; e < TILE2; e += FB) L[e / TILE][e % TILE] = tp[e];
  __syncthreads();
  for (int j = 0; j < TILE; ++j) {
    if (threadIdx.x == 0) {
      T dj = L[j][j];
      if (!(dj > T(0))) {
        if (atomicCAS(&err->code, 0, (int)SFCDD_ERR_NOT_SPD) == 0) err->index = m;
        dj = T(1);
      }
      const T piv = sqrt(dj);
      L[j][j] = piv;
      s_inv = T(1) / piv;
    }
    __syncthreads();
    const T inv = s_inv;
    for (int i = j + 1 + threadIdx.x; i < TILE; i += FB) L[i][j] *= inv;
    __syncthreads();
    const int rem = TILE - j - 1;
    for (int e = threadIdx.x; e < rem * rem; e += FB) {
      const int i = j + 1 + e / rem, l = j + 1 + e % rem;
      if (l <= i) L[i][l] -= L[i][j] * L[l][j];
    }
    __syncthreads();
  }
  // inverse of the lower-triangular block, one column per thread
  if (threadIdx.x < TILE) {
    const int c = threadIdx.x;
    for (int i = 0; i < c; ++i) X[i][c] = T(0);
    for (int i = c; i < TILE; ++i) {
      T s = (i == c) ? T(1) : T(0);
      for (int kk = c; kk < i; ++kk) s -= L[i][kk] * X[kk][c];
      X[i][c] = s / L[i][i];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TILE2; e += FB) tp[e] = X[e / TILE][e % TILE];
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

// Panel: L_ik = A_ik * Linv_kk^T for every tile row i > k.  grid = (max rows, nmat)
template <class T>
__global__ void __launch_bounds__(FB) k_trsm(TileSetDev ts, int mat0, int k, T* __restrict__ tiles) {
  extern __shared__ __align__(16) unsigned char dsm_trsm[];
  T (*At)[TILE + 4] = reinterpret_cast<T (*)[TILE + 4]>(dsm_trsm);
  T (*Bt)[TILE + 4] = At + TILE;
  const int m = mat0 + blockIdx.y;
  const int nt = ts.nt[m];
  const int i = k + 1 + blockIdx.x;
  if (i >= nt) return;
  T* base = tiles + ts.tbase[m];
  T* aik = base + (long long)(i * (i + 1) / 2 + k) * TILE2;
  const T* lkk = base + (long long)(k * (k + 1) / 2 + k) * TILE2;
  load_transposed<T>(At, aik);
  load_transposed<T>(Bt, lkk);
  __syncthreads();
  const int r0 = (threadIdx.x / 16) * 4, c0 = (threadIdx.x % 16) * 4;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  mma_4x4<T>(acc, At, Bt, r0, c0);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) aik[(r0 + a) * TILE + c0 + b] = acc[a][b];
}

// Trailing update A_ij -= L_ik L_jk^T for k < j <= i.  grid = (pairs, nmat)
template <class T>
__global__ void __launch_bounds__(FB) k_syrk(TileSetDev ts, int mat0, int k, T* __restrict__ tiles) {
  extern __shared__ __align__(16) unsigned char dsm_syrk[];
  T (*Xt)[TILE + 4] = reinterpret_cast<T (*)[TILE + 4]>(dsm_syrk);
  T (*Yt)[TILE + 4] = Xt + TILE;
  const int m = mat0 + blockIdx.y;
  const int nt = ts.nt[m];
  const int rem = nt - k - 1;
  if ((int)blockIdx.x >= rem * (rem + 1) / 2) return;
  int ii, jj;
  tri_decode(blockIdx.x, ii, jj);
  const int i = k + 1 + ii, j = k + 1 + jj;
  T* base = tiles + ts.tbase[m];
  const T* lik = base + (long long)(i * (i + 1) / 2 + k) * TILE2;
  const T* ljk = base + (long long)(j * (j + 1) / 2 + k) * TILE2;
  T* aij = base + (long long)(i * (i + 1) / 2 + j) * TILE2;
  load_transposed<T>(Xt, lik);
  load_transposed<T>(Yt, ljk);
  __syncthreads();
  const int r0 = (threadIdx.x / 16) * 4, c0 = (threadIdx.x % 16) * 4;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  mma_4x4<T>(acc, Xt, Yt, r0, c0);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) aij[(r0 + a) * TILE + c0 + b] -= acc[a][b];
}

template <class T>
static void factor_tiles_t(const TileSetDev& ts, int mat0, int nmat, int max_nt, T* tiles,
                           ErrWord* err, cudaStream_t s, LaunchHook* hook) {
  const int sm_potrf = (2 * TILE + 1) * (TILE + 1) * (int)sizeof(T);
  const int sm_gemm = 2 * TILE * (TILE + 4) * (int)sizeof(T);
  cudaFuncSetAttribute(k_potrf<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_potrf);
  cudaFuncSetAttribute(k_trsm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_gemm);
  cudaFuncSetAttribute(k_syrk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_gemm);
  for (int k = 0; k < max_nt; ++k) {
    hook->before(SFCDD_K_POTRF);
    k_potrf<T><<<nmat, FB, sm_potrf, s>>>(ts, mat0, k, tiles, err);
    hook->after(SFCDD_K_POTRF);
    const int rows = max_nt - k - 1;
    if (rows > 0) {
      hook->before(SFCDD_K_TRSM);
      k_trsm<T><<<dim3(rows, nmat), FB, sm_gemm, s>>>(ts, mat0, k, tiles);
      hook->after(SFCDD_K_TRSM);
      hook->before(SFCDD_K_SYRK);
      k_syrk<T><<<dim3(rows * (rows + 1) / 2, nmat), FB, sm_gemm, s>>>(ts, mat0, k, tiles);
      hook->after(SFCDD_K_SYRK);
    }
  }
}

void factor_tiles(const TileSetDev& ts, int mat0, int nmat, int max_nt, void* tiles, Store st,
                  ErrWord* err, cudaStream_t s, LaunchHook* hook) {
  if (st == Store::F64)
    factor_tiles_t<double>(ts, mat0, nmat, max_nt, (double*)tiles, err, s, hook);
  else
    factor_tiles_t<float>(ts, mat0, nmat, max_nt, (float*)tiles, err, s, hook);
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

// Dense symmetric N x N copy (row-major) of an FP64 packed matrix before
// factorization (introspection only).
__global__ void k_unpack_dense(TileSetDev ts, int m, const double* __restrict__ tiles,
                               double* __restrict__ dense) {
  const int n = ts.n[m];
  const long long tot = (long long)n * n;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += stride) {
    int r = (int)(e / n), c = (int)(e % n);
    if (c > r) {
      const int t = r;
      r = c;
      c = t;
    }
    const int a = r / TILE, b = c / TILE;
    dense[e] = tiles[ts.tbase[m] + (long long)(a * (a + 1) / 2 + b) * TILE2 + (r % TILE) * TILE +
                     (c % TILE)];
  }
}

void launch_unpack_dense(const TileSetDev& ts, int m, const double* tiles, double* dense,
                         cudaStream_t s) {
  k_unpack_dense<<<152 * 8, 256, 0, s>>>(ts, m, tiles, dense);
}

}  // namespace sfcdd
