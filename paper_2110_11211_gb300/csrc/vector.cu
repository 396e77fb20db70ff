// Curve-order vector kernels of one PCG iteration: the matrix-free stencil
// (Sec. 4 operator), the fused PCG updates and reductions (Sec. 3.3, PCG), the
// coarse restriction R_0 (eq. restr) and the prolongation with the
// partition-of-unity weights (eq. addSW, Algorithm 2 step 4).
//
// Reductions are deterministic: a fixed grid (a function of N only) assigns
// every element to one block, each block writes its partial, and the last
// block to arrive sums the partials in block order and updates the scalars.
// FP64 adds issue at 1/64 of the FP32 rate on this GPU, so the shuffle trees of
// the reductions cost as much as the element arithmetic unless every thread
// first accumulates several elements: kernels that reduce run on at most two
// blocks per SM (about four elements per thread).
#include <algorithm>

#include "device_common.cuh"

namespace sfcdd {

constexpr int VB = 256;                 // threads per block of vector kernels
constexpr int VMAXBLOCKS = 152 * 8;     // grid cap (8 blocks per SM)
constexpr int RMAXBLOCKS = 152 * 2;     // grid cap of kernels that reduce
constexpr int RPER = 4;                 // elements per thread they aim for

int vec_blocks(int n) {
  int b = (n + VB - 1) / VB;
  if (b > VMAXBLOCKS) b = VMAXBLOCKS;
  if (b < 1) b = 1;
  return b;
}

int red_blocks(int n) {
  int b = (n + VB * RPER - 1) / (VB * RPER);
  if (b > RMAXBLOCKS) b = RMAXBLOCKS;
  if (b < 1) b = 1;
  return b;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduce K values, store the block partial, and let the last block call
// fin(totals).  Must be reached by every thread of every block of the grid.
// K <= 2 (the PCG reductions): with two values the first warp exchange halves
// the work (lanes 0-15 keep value 0, lanes 16-31 value 1), so a warp pays five
// FP64 adds instead of ten; the eight warp partials of both values then go
// through one three-level tree (value k of warp u in lane 8 k + u).
template <int K, class Fin>
__device__ __forceinline__ void reduce_finalize(double (&v)[K], ReduceWs ws, Fin fin) {
  constexpr int NW = VB / 32;
  static_assert(NW == 8, "eight warps per block");
  __shared__ double sh[K][NW];
  __shared__ bool is_last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if constexpr (K <= 2) {
    double t;
    int o = 16;
    if constexpr (K == 2) {
      const bool hi = (lane & 16) != 0;
      const double keep = hi ? v[1] : v[0], send = hi ? v[0] : v[1];
      t = keep + __shfl_xor_sync(0xffffffffu, send, 16);
      o = 8;
    } else {
      t = v[0];
    }
    for (; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((lane & 15) == 0 && (lane >> 4) < K) sh[lane >> 4][w] = t;
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const double s = warp_sum(v[k]);
      if (lane == 0) sh[k][w] = s;
    }
  }
  __syncthreads();
  if (w == 0) {
    if constexpr (K <= 2) {
      const int k = lane >> 3, u = lane & 7;
      double s = k < K ? sh[k][u] : 0.0;
      s += __shfl_xor_sync(0xffffffffu, s, 4);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      if (u == 0 && k < K) ws.partial[blockIdx.x * K + k] = s;
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        double s = lane < NW ? sh[k][lane] : 0.0;
        s = warp_sum(s);
        if (lane == 0) ws.partial[blockIdx.x * K + k] = s;
      }
    }
    if (lane == 0) {
      __threadfence();
      const unsigned t = atomicAdd(ws.counter, 1u);
      is_last = (t == gridDim.x - 1);
    }
  }
  __syncthreads();
  if (is_last && w == 0) {
    __threadfence();
    double tot[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(&ws.partial[b * K + k]);
      tot[k] = warp_sum(s);
    }
    if (lane == 0) {
      fin(tot);
      *ws.counter = 0u;
      __threadfence();
    }
  }
}

// ---------------------------------------------------------------------------
// Stencil y = A x in curve order.  Neighbours: the point's packed code gives
// its coordinates; code +- 2^{off_j} is the axis-j neighbour, whose curve
// position comes from invpad.  MODE 0: y = A x; 1: also p^T A p -> alpha;
// 2: y = b - A x and ||y|| -> true relative residual; 3: y = b - A x.  MODE 0
// and 3 with sc != null return once the solve has converged.
template <int D, int MODE>
__global__ void __launch_bounds__(VB) k_stencil(GridDev g, const unsigned* __restrict__ code,
                                                const int* __restrict__ invpad,
                                                const double* __restrict__ x,
                                                double* __restrict__ y,
                                                const double* __restrict__ b, PcgScalars* sc,
                                                ReduceWs ws) {
  if ((MODE == 1 || ((MODE == 0 || MODE == 3) && sc)) && sc->done) return;
  double acc = 0.0;
  const int stride = gridDim.x * VB;
#pragma unroll 4
  for (int p = blockIdx.x * VB + threadIdx.x; p < g.N; p += stride) {
    double xc;
    double v = stencil_point<D>(g, code, invpad, x, p, xc);
    if (MODE == 2) {
      v = b[p] - v;
      acc += v * v;
    } else if (MODE == 3) {
      v = b[p] - v;
    } else if (MODE == 1) {
      acc += xc * v;
    }
    y[p] = v;
  }
  if (MODE == 1) {
    double vv[1] = {acc};
    reduce_finalize<1>(vv, ws, [&](double* t) {
      sc->pq = t[0];
      sc->alpha = sc->rz / t[0];
      if (sc->hist_alpha && sc->iter < sc->hist_cap) sc->hist_alpha[sc->iter] = sc->alpha;
    });
  } else if (MODE == 2) {
    double vv[1] = {acc};
    reduce_finalize<1>(vv, ws, [&](double* t) {
      sc->true_rel = sc->bb > 0.0 ? sqrt(t[0] / sc->bb) : 0.0;
    });
  }
}

template <int MODE>
static void stencil_dispatch(const GridDev& g, const unsigned* code, const int* invpad,
                             const double* x, double* y, const double* b, PcgScalars* sc,
                             ReduceWs ws, cudaStream_t s) {
  const int nb = (MODE == 1 || MODE == 2) ? red_blocks(g.N) : vec_blocks(g.N);
  switch (g.d) {
    case 1: k_stencil<1, MODE><<<nb, VB, 0, s>>>(g, code, invpad, x, y, b, sc, ws); break;
    case 2: k_stencil<2, MODE><<<nb, VB, 0, s>>>(g, code, invpad, x, y, b, sc, ws); break;
    case 3: k_stencil<3, MODE><<<nb, VB, 0, s>>>(g, code, invpad, x, y, b, sc, ws); break;
    case 4: k_stencil<4, MODE><<<nb, VB, 0, s>>>(g, code, invpad, x, y, b, sc, ws); break;
    case 5: k_stencil<5, MODE><<<nb, VB, 0, s>>>(g, code, invpad, x, y, b, sc, ws); break;
    case 6: k_stencil<6, MODE><<<nb, VB, 0, s>>>(g, code, invpad, x, y, b, sc, ws); break;
    case 7: k_stencil<7, MODE><<<nb, VB, 0, s>>>(g, code, invpad, x, y, b, sc, ws); break;
    default: k_stencil<8, MODE><<<nb, VB, 0, s>>>(g, code, invpad, x, y, b, sc, ws); break;
  }
}

void launch_stencil(const GridDev& g, const unsigned* code, const int* invpad, const double* x,
                    double* y, int mode, PcgScalars* sc, ReduceWs ws, cudaStream_t s) {
  if (mode == 1)
    stencil_dispatch<1>(g, code, invpad, x, y, nullptr, sc, ws, s);
  else
    stencil_dispatch<0>(g, code, invpad, x, y, nullptr, sc, ws, s);
}

void launch_residual(const GridDev& g, const unsigned* code, const int* invpad, const double* b,
                     const double* x, double* y, PcgScalars* sc, ReduceWs ws, cudaStream_t s) {
  stencil_dispatch<3>(g, code, invpad, x, y, b, sc, ws, s);
}

void launch_true_residual(const GridDev& g, const unsigned* code, const int* invpad,
                          const double* b, const double* x, double* tmp, PcgScalars* sc,
                          ReduceWs ws, cudaStream_t s) {
  stencil_dispatch<2>(g, code, invpad, x, tmp, b, sc, ws, s);
}

// ---------------------------------------------------------------------------
// x += alpha p, r -= alpha q, ||r||^2 -> convergence test.
__global__ void __launch_bounds__(VB) k_update_xr(int n, double* __restrict__ x,
                                                  double* __restrict__ r,
                                                  const double* __restrict__ p,
                                                  const double* __restrict__ q, PcgScalars* sc,
                                                  ReduceWs ws) {
  if (sc->done) return;
  const double alpha = sc->alpha;
  double acc[2] = {0.0, 0.0};
  const int stride = gridDim.x * VB;
#pragma unroll 4
  for (int i = blockIdx.x * VB + threadIdx.x; i < n; i += stride) {
    const double xi = x[i] + alpha * p[i];
    x[i] = xi;
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    acc[0] += ri * ri;
    acc[1] += xi * ri;
  }
  reduce_finalize<2>(acc, ws, [&](double* t) {
    sc->rr = t[0];
    // energy mode (f = 0): ||x||_A / ||x_0||_A with ||x||_A^2 = -x^T r
    const double rel = sc->energy ? sqrt(fmax(-t[1], 0.0) / sc->esq0) : sqrt(t[0] / sc->bb);
    sc->rel = rel;
    sc->iter += 1;
    if (!(rel == rel) || isinf(rel) || !(sc->alpha == sc->alpha) || isinf(sc->alpha)) {
      sc->status = SFCDD_ERR_NAN;
      sc->done = 1;
    } else if (rel <= sc->rtol) {
      sc->done = 1;
    }
  });
}

void launch_update_xr(int n, double* x, double* r, const double* p, const double* q,
                      PcgScalars* sc, ReduceWs ws, cudaStream_t s) {
  k_update_xr<<<red_blocks(n), VB, 0, s>>>(n, x, r, p, q, sc, ws);
}

// Energy-norm protocol (f = 0): r = -A x is given; init = 1 resets the PCG
// scalars with ||x_0||_A^2 = -x^T r, otherwise sc->true_rel = ||x||_A / ||x_0||_A.
__global__ void __launch_bounds__(VB) k_energy(int n, const double* __restrict__ x,
                                               const double* __restrict__ r, PcgScalars* sc,
                                               ReduceWs ws, double rtol, int flexible, int init) {
  double acc = 0.0;
  const int stride = gridDim.x * VB;
#pragma unroll 4
  for (int i = blockIdx.x * VB + threadIdx.x; i < n; i += stride) acc += x[i] * r[i];
  double vv[1] = {acc};
  reduce_finalize<1>(vv, ws, [&](double* t) {
    const double esq = fmax(-t[0], 0.0);
    if (init) {
      sc->esq0 = esq;
      sc->energy = 1;
      sc->bb = 1.0;
      sc->rr = 0.0;
      sc->rel = esq > 0.0 ? 1.0 : 0.0;
      sc->true_rel = sc->rel;
      sc->rz = 0.0;
      sc->rz_old = 0.0;
      sc->pq = 0.0;
      sc->alpha = 0.0;
      sc->beta = 0.0;
      sc->iter = 0;
      sc->status = 0;
      sc->rtol = rtol;
      sc->flexible = flexible;
      sc->done = esq > 0.0 ? 0 : 1;
      if (!(t[0] == t[0]) || isinf(t[0])) {  // non-finite initial iterate
        sc->status = SFCDD_ERR_NAN;
        sc->done = 1;
      }
    } else {
      sc->true_rel = sc->esq0 > 0.0 ? sqrt(esq / sc->esq0) : 0.0;
    }
  });
}

void launch_energy(int n, const double* x, const double* r, PcgScalars* sc, ReduceWs ws,
                   double rtol, int flexible, int init, cudaStream_t s) {
  k_energy<<<red_blocks(n), VB, 0, s>>>(n, x, r, sc, ws, rtol, flexible, init);
}

// ---------------------------------------------------------------------------
// Coarse right-hand side g0 = R_0 r (eq. restr): eight lanes per coarse block
// (blocks hold N / (q P) points, a few dozen at the paper's q), summed by a
// fixed three-level tree.
constexpr int RL = 8;
__global__ void k_restrict(PartDev pd, const double* __restrict__ r, double* __restrict__ g0,
                           const PcgScalars* sc) {
  if (sc && sc->done) return;
  const int l = threadIdx.x & (RL - 1);
  const int a = (blockIdx.x * blockDim.x + threadIdx.x) / RL;
  const int N0 = pd.q * pd.P;
  const bool valid = a < N0;  // partial warps stay for the shuffles
  double s = 0.0;
  if (valid) {
    const int t = a / pd.q, m = a % pd.q;
    const int n = tilde_size(pd, t);
    const int bf = n / pd.q, br = n % pd.q;
    const int start = tilde_off(pd, t) + (m < br ? m * (bf + 1) : br * (bf + 1) + (m - br) * bf);
    const int size = m < br ? bf + 1 : bf;
    for (int k = l; k < size; k += RL) s += r[start + k];
  }
  s += __shfl_xor_sync(0xffffffffu, s, 4);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  if (valid && l == 0) g0[a] = s;
}

void launch_restrict(const PartDev& pd, const double* r, double* g0, const PcgScalars* sc,
                     cudaStream_t s) {
  const long long threads = (long long)pd.q * pd.P * RL;
  k_restrict<<<(unsigned)((threads + VB - 1) / VB), VB, 0, s>>>(pd, r, g0, sc);
}

// ---------------------------------------------------------------------------
// Prolongation z = R_0^T d_0 + sum_i omega_i R_i^T d_i (eq. addSW), gathered
// per curve position from the (at most min(2g+3, P)) subdomains whose range can
// contain it; fused with r^T z (and r^T z_old for the flexible beta).
// mode: 0 additive two-level, 1 one level, 2 coarse only.  DOT: PCG finalize.
// The PCG finalize of r^T z: beta (Hestenes-Stiefel, or Polak-Ribiere for the
// flexible variant) from t = {r^T z_new, r^T z_old}.
__device__ __forceinline__ void finalize_rz(PcgScalars* sc, const double* t) {
  const double rz_new = t[0];
  if (sc->iter == 0) {
    sc->beta = 0.0;
  } else if (sc->flexible) {
    sc->beta = (rz_new - t[1]) / sc->rz;
  } else {
    sc->beta = rz_new / sc->rz;
  }
  sc->rz_old = t[1];
  sc->rz = rz_new;
  // beta_k (p_{k+1} = z_{k+1} + beta_k p_k) after update k (iter = k + 1)
  if (sc->hist_beta && sc->iter >= 1 && sc->iter - 1 < sc->hist_cap)
    sc->hist_beta[sc->iter - 1] = sc->beta;
}

// sc != null without DOT: only the early return once the solve has converged.
template <bool DOT>
__global__ void __launch_bounds__(VB) k_prolong(PartDev pd, TileSetDev ts, int mode,
                                                const double* __restrict__ dvec,
                                                const double* __restrict__ r,
                                                double* __restrict__ z, PcgScalars* sc,
                                                ReduceWs ws) {
  if (sc && sc->done) return;
  double acc[2] = {0.0, 0.0};
  const int stride = gridDim.x * VB;
  const int coarse_base = mode != 1 ? __ldg(&ts.vbase[pd.P]) : 0;
  auto lvbase = [&](int i) { return __ldg(&ts.vbase[i]); };
  for (int p = blockIdx.x * VB + threadIdx.x; p < pd.N; p += stride) {
    const double v = prolong_point(pd, mode, dvec, coarse_base, lvbase, ts.linv, p);
    if (DOT) {
      const double rp = r[p];
      acc[0] += rp * v;
      acc[1] += rp * z[p];
    }
    z[p] = v;
  }
  if (DOT) reduce_finalize<2>(acc, ws, [&](double* t) { finalize_rz(sc, t); });
}

void launch_prolong(const PartDev& pd, const TileSetDev& ts, int mode, const double* dvec,
                    const double* r, double* z, PcgScalars* sc, ReduceWs ws, cudaStream_t s,
                    bool dot) {
  if (sc && dot)
    // one point per thread: its gathers are dependent loads, which more points per
    // thread would serialize
    k_prolong<true><<<vec_blocks(pd.N), VB, 0, s>>>(pd, ts, mode, dvec, r, z, sc, ws);
  else
    k_prolong<false><<<vec_blocks(pd.N), VB, 0, s>>>(pd, ts, mode, dvec, r, z, sc, ws);
}

// Balanced operator (eq. balSW) from its parts: z = t - v + w with w = F g,
// t = C_(1) (g - A w), v = F A t; with sc: the PCG finalize of r^T z as in the
// prolongation.
template <bool DOT>
__global__ void __launch_bounds__(VB) k_combine_bal(int n, const double* __restrict__ t,
                                                    const double* __restrict__ v,
                                                    const double* __restrict__ w,
                                                    const double* __restrict__ r,
                                                    double* __restrict__ z, PcgScalars* sc,
                                                    ReduceWs ws) {
  if (DOT && sc->done) return;
  double acc[2] = {0.0, 0.0};
  const int stride = gridDim.x * VB;
#pragma unroll 4
  for (int p = blockIdx.x * VB + threadIdx.x; p < n; p += stride) {
    const double zp = (t[p] - v[p]) + w[p];
    if (DOT) {
      const double rp = r[p];
      acc[0] += rp * zp;
      acc[1] += rp * z[p];
    }
    z[p] = zp;
  }
  if (DOT) reduce_finalize<2>(acc, ws, [&](double* tt) { finalize_rz(sc, tt); });
}

void launch_combine_bal(int n, const double* t, const double* v, const double* w, const double* r,
                        double* z, PcgScalars* sc, ReduceWs ws, cudaStream_t s) {
  if (sc)
    k_combine_bal<true><<<red_blocks(n), VB, 0, s>>>(n, t, v, w, r, z, sc, ws);
  else
    k_combine_bal<false><<<vec_blocks(n), VB, 0, s>>>(n, t, v, w, r, z, sc, ws);
}

// p = z + beta p
__global__ void __launch_bounds__(VB) k_update_p(int n, const double* __restrict__ z,
                                                 double* __restrict__ p, const PcgScalars* sc) {
  if (sc->done) return;
  const double beta = sc->beta;
  const int stride = gridDim.x * VB;
  for (int i = blockIdx.x * VB + threadIdx.x; i < n; i += stride) p[i] = z[i] + beta * p[i];
}

void launch_update_p(int n, const double* z, double* p, const PcgScalars* sc, cudaStream_t s) {
  k_update_p<<<vec_blocks(n), VB, 0, s>>>(n, z, p, sc);
}

// x = 0, r = b, p = 0, ||b||^2 and reset of the PCG scalars.
__global__ void __launch_bounds__(VB) k_init_pcg(int n, const double* __restrict__ b,
                                                 double* __restrict__ x, double* __restrict__ r,
                                                 PcgScalars* sc, ReduceWs ws, double rtol,
                                                 int flexible) {
  double acc = 0.0;
  const int stride = gridDim.x * VB;
#pragma unroll 4
  for (int i = blockIdx.x * VB + threadIdx.x; i < n; i += stride) {
    const double bi = b[i];
    x[i] = 0.0;
    r[i] = bi;
    acc += bi * bi;
  }
  double vv[1] = {acc};
  reduce_finalize<1>(vv, ws, [&](double* t) {
    sc->energy = 0;
    sc->bb = t[0];
    sc->rr = t[0];
    sc->rel = t[0] > 0.0 ? 1.0 : 0.0;
    sc->rz = 0.0;
    sc->rz_old = 0.0;
    sc->pq = 0.0;
    sc->alpha = 0.0;
    sc->beta = 0.0;
    sc->iter = 0;
    sc->status = 0;
    sc->rtol = rtol;
    sc->flexible = flexible;
    sc->done = t[0] > 0.0 ? 0 : 1;
    if (!(t[0] == t[0]) || isinf(t[0])) {  // non-finite right-hand side
      sc->status = SFCDD_ERR_NAN;
      sc->done = 1;
    }
  });
}

void launch_init_pcg(int n, const double* b, double* x, double* r, PcgScalars* sc, ReduceWs ws,
                     double rtol, int flexible, cudaStream_t s) {
  k_init_pcg<<<red_blocks(n), VB, 0, s>>>(n, b, x, r, sc, ws, rtol, flexible);
}

__global__ void k_axpby(int n, double a, const double* __restrict__ x, double b,
                        const double* __restrict__ y, double* __restrict__ out) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

void launch_axpby(int n, double a, const double* x, double b, const double* y, double* out,
                  cudaStream_t s) {
  k_axpby<<<vec_blocks(n), VB, 0, s>>>(n, a, x, b, y, out);
}

// ---------------------------------------------------------------------------
// Permutations between the caller's lexicographic order and curve order.
__device__ __forceinline__ int lex_id(const GridDev& g, unsigned c) {
  int id = 0;
  for (int j = 0; j < g.d; ++j) {
    const int kj = (int)((c >> g.off[j]) & ((1u << g.lev[j]) - 1u));
    id += (kj - 1) * g.stride[j];
  }
  return id;
}

__global__ void k_lex_to_curve(GridDev g, const unsigned* __restrict__ code,
                               const double* __restrict__ in, double* __restrict__ out) {
  const int stride = gridDim.x * blockDim.x;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < g.N; p += stride)
    out[p] = in[lex_id(g, code[p])];
}

__global__ void k_curve_to_lex(GridDev g, const unsigned* __restrict__ code,
                               const double* __restrict__ in, double* __restrict__ out) {
  const int stride = gridDim.x * blockDim.x;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < g.N; p += stride)
    out[lex_id(g, code[p])] = in[p];
}

void launch_lex_to_curve(const GridDev& g, const unsigned* code, const double* in, double* out,
                         cudaStream_t s) {
  k_lex_to_curve<<<vec_blocks(g.N), VB, 0, s>>>(g, code, in, out);
}
void launch_curve_to_lex(const GridDev& g, const unsigned* code, const double* in, double* out,
                         cudaStream_t s) {
  k_curve_to_lex<<<vec_blocks(g.N), VB, 0, s>>>(g, code, in, out);
}

// ---------------------------------------------------------------------------
// dL/dc_j = -sum_p lambda_p 4^{l_j} (2 u_p - u_{p-e_j} - u_{p+e_j}), all j in one pass.
template <int D>
__global__ void __launch_bounds__(VB) k_grad(GridDev g, const unsigned* __restrict__ code,
                                             const int* __restrict__ invpad,
                                             const double* __restrict__ lam,
                                             const double* __restrict__ u, PcgScalars* sc,
                                             ReduceWs ws) {
  double acc[D];
#pragma unroll
  for (int j = 0; j < D; ++j) acc[j] = 0.0;
  const int stride = gridDim.x * VB;
  for (int p = blockIdx.x * VB + threadIdx.x; p < g.N; p += stride) {
    const unsigned c = code[p];
    const double up = u[p], lp = lam[p];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const unsigned kj = (c >> g.off[j]) & ((1u << g.lev[j]) - 1u);
      const unsigned unit = 1u << g.off[j];
      double v = 2.0 * up;
      if (kj > 1u) v -= u[invpad[c - unit]];
      if (kj < (unsigned)g.size[j]) v -= u[invpad[c + unit]];
      acc[j] += lp * v;
    }
  }
  reduce_finalize<D>(acc, ws, [&](double* t) {
    for (int j = 0; j < D; ++j) sc->grad[j] = -ldexp(t[j], 2 * g.lev[j]);
  });
}

void launch_grad(const GridDev& g, const unsigned* code, const int* invpad, const double* lam,
                 const double* u, PcgScalars* sc, ReduceWs ws, cudaStream_t s) {
  const int nb = vec_blocks(g.N);
  switch (g.d) {
    case 1: k_grad<1><<<nb, VB, 0, s>>>(g, code, invpad, lam, u, sc, ws); break;
    case 2: k_grad<2><<<nb, VB, 0, s>>>(g, code, invpad, lam, u, sc, ws); break;
    case 3: k_grad<3><<<nb, VB, 0, s>>>(g, code, invpad, lam, u, sc, ws); break;
    case 4: k_grad<4><<<nb, VB, 0, s>>>(g, code, invpad, lam, u, sc, ws); break;
    case 5: k_grad<5><<<nb, VB, 0, s>>>(g, code, invpad, lam, u, sc, ws); break;
    case 6: k_grad<6><<<nb, VB, 0, s>>>(g, code, invpad, lam, u, sc, ws); break;
    case 7: k_grad<7><<<nb, VB, 0, s>>>(g, code, invpad, lam, u, sc, ws); break;
    default: k_grad<8><<<nb, VB, 0, s>>>(g, code, invpad, lam, u, sc, ws); break;
  }
}

// ---------------------------------------------------------------------------
// The vector phase of one PCG iteration as one cooperative launch.  Between
// the backward substitution of iteration k and the forward substitution of
// iteration k + 1 the iteration needs, in order: the prolongation z (eq. addSW)
// with r^T z (beta), p = z + beta p with q = A p (alpha), the x / r update with
// ||r|| (convergence), and the coarse restriction R_0 r (eq. restr) of the next
// preconditioner apply.  As separate launches these are five kernels whose
// time goes to latency (dependent gathers, reductions through the last CTA),
// not to bytes or FP64 work; here every CTA owns a fixed range of curve
// positions through all three phases and the two scalars a later phase needs
// (beta, alpha) are exchanged through two grid barriers.  Every CTA sums the
// block partials itself, in the same fixed order, so all of them obtain
// bit-identical scalars without a second barrier; CTA 0 publishes them.
// The stencil reads p_new = z + beta p_old at the neighbours on the fly (z is
// complete after the first barrier), so p needs no barrier of its own: p of
// the previous iteration stays in one buffer and the new p goes to the other.
namespace {

constexpr int FB_THREADS = 256;
constexpr long long BAR_SPIN_LIMIT = 1ll << 24;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier of a cooperative launch (all CTAs resident).  One arrival
// counter that only grows during a solve (reset when the solve starts): the
// b-th barrier of iteration `iter` releases once the counter reaches
// (2 iter + b + 1) nblocks, so arriving is one fire-and-forget release add and
// waiting one acquire poll, with no reset on the critical path.  Bounded: a
// timeout records TIMEOUT (site 30) and lets the CTA go on, so the launch
// always ends.
__device__ __forceinline__ void grid_barrier(unsigned* count, unsigned target, ErrWord* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
    long long it = 0;
    while ((int)(ld_acquire_u32(count) - target) < 0) {
      if (++it > 256) __nanosleep(20);
      if (it > BAR_SPIN_LIMIT) {
        if (atomicCAS(&err->code, 0, (int)SFCDD_ERR_TIMEOUT) == 0) err->index = 30;
        break;
      }
    }
  }
  __syncthreads();
}

// Block sum of two values (every thread passes its pair; thread 0 gets totals).
__device__ __forceinline__ void block_sum2(double& a, double& b, double (*sh)[FB_THREADS / 32]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool hi = (lane & 16) != 0;
  double t = (hi ? b : a) + __shfl_xor_sync(0xffffffffu, hi ? a : b, 16);
  for (int o = 8; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((lane & 15) == 0) sh[lane >> 4][w] = t;
  __syncthreads();
  if (w == 0) {
    const int k = lane >> 3, u = lane & 7;
    double v = k < 2 ? sh[k][u] : 0.0;
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    a = __shfl_sync(0xffffffffu, v, 0);
    b = __shfl_sync(0xffffffffu, v, 8);
  }
}

// Totals of the two block partials of a phase over all CTAs, summed by warp 0
// of every CTA in the same order (bit-identical in every CTA); broadcast to
// the CTA through shared memory.
__device__ __forceinline__ void grid_totals(const double* part, int nblocks, double* out2) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 32) {
    double s0 = 0.0, s1 = 0.0;
    for (int b = lane; b < nblocks; b += 32) {
      s0 += __ldcg(&part[2 * b]);
      s1 += __ldcg(&part[2 * b + 1]);
    }
    for (int o = 16; o > 0; o >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if (lane == 0) {
      out2[0] = s0;
      out2[1] = s1;
    }
  }
  __syncthreads();
}

template <int D>
__global__ void __launch_bounds__(FB_THREADS) k_pcg_fused(FusedPcg a) {
  __shared__ double sh[2][FB_THREADS / 32];
  __shared__ double tot[2];
  PcgScalars* sc = a.sc;
  // scalars of the previous iteration, read before anything is published
  if (sc->done) return;  // uniform: nothing writes done before the last phase
  const int iter = sc->iter;
  const double rz_prev = sc->rz;
  const int flexible = sc->flexible;
  const int c = blockIdx.x;
  const int lo = a.range[c], hi = a.range[c + 1];
  const double* pold = a.p[iter & 1];
  double* pnew = a.p[(iter + 1) & 1];

  // phase 1: z = C^{-1} r from the substitution results, r^T z and r^T z_old
  double acc0 = 0.0, acc1 = 0.0;
  {
    const int coarse_base = a.mode != 1 ? __ldg(&a.ts.vbase[a.pd.P]) : 0;
    auto lvbase = [&](int i) { return __ldg(&a.ts.vbase[i]); };
    for (int p = lo + threadIdx.x; p < hi; p += FB_THREADS) {
      const double v = prolong_point(a.pd, a.mode, a.dvec, coarse_base, lvbase, a.ts.linv, p);
      const double rp = a.r[p];
      acc0 += rp * v;
      acc1 += rp * a.z[p];
      a.z[p] = v;
    }
  }
  block_sum2(acc0, acc1, sh);
  if (threadIdx.x == 0) {
    a.part[2 * c] = acc0;
    a.part[2 * c + 1] = acc1;
  }
  grid_barrier(a.bar, (unsigned)(2 * iter + 1) * (unsigned)a.nblocks, a.err);
  grid_totals(a.part, a.nblocks, tot);
  const double rz = tot[0], rz_oldz = tot[1];
  const double beta = iter == 0 ? 0.0 : (flexible ? (rz - rz_oldz) / rz_prev : rz / rz_prev);
  if (c == 0 && threadIdx.x == 0) {
    sc->beta = beta;
    sc->rz_old = rz_oldz;
    sc->rz = rz;
    if (sc->hist_beta && iter >= 1 && iter - 1 < sc->hist_cap) sc->hist_beta[iter - 1] = beta;
  }

  // phase 2: p_new = z + beta p_old (neighbours on the fly), q = A p_new, p^T q
  double pq = 0.0;
  for (int p = lo + threadIdx.x; p < hi; p += FB_THREADS) {
    const unsigned cd = __ldg(&a.code[p]);
    // z was written by other CTAs of this launch: read it through L2 (__ldcg)
    const double pc = __ldcg(&a.z[p]) + beta * pold[p];
    double v = a.g.diag * pc;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const unsigned kj = (cd >> a.g.off[j]) & ((1u << a.g.lev[j]) - 1u);
      const unsigned unit = 1u << a.g.off[j];
      if (kj > 1u) {
        const int n = __ldg(&a.invpad[cd - unit]);
        v -= a.g.w[j] * (__ldcg(&a.z[n]) + beta * pold[n]);
      }
      if (kj < (unsigned)a.g.size[j]) {
        const int n = __ldg(&a.invpad[cd + unit]);
        v -= a.g.w[j] * (__ldcg(&a.z[n]) + beta * pold[n]);
      }
    }
    pnew[p] = pc;
    a.q[p] = v;
    pq += pc * v;
  }
  double dummy = 0.0;
  block_sum2(pq, dummy, sh);
  if (threadIdx.x == 0) {
    a.part[2 * (a.nblocks + c)] = pq;
    a.part[2 * (a.nblocks + c) + 1] = 0.0;
  }
  grid_barrier(a.bar, (unsigned)(2 * iter + 2) * (unsigned)a.nblocks, a.err);
  grid_totals(a.part + 2 * a.nblocks, a.nblocks, tot);
  const double pq_tot = tot[0];
  const double alpha = rz / pq_tot;
  if (c == 0 && threadIdx.x == 0) {
    sc->pq = pq_tot;
    sc->alpha = alpha;
    if (sc->hist_alpha && iter < sc->hist_cap) sc->hist_alpha[iter] = alpha;
  }

  // phase 3: x += alpha p, r -= alpha q, ||r||^2 and x^T r (energy); then the
  // coarse restriction of the new r over this CTA's whole coarse blocks
  double rr = 0.0, xr = 0.0;
  for (int p = lo + threadIdx.x; p < hi; p += FB_THREADS) {
    const double xi = a.x[p] + alpha * pnew[p];
    a.x[p] = xi;
    const double ri = a.r[p] - alpha * a.q[p];
    a.r[p] = ri;
    rr += ri * ri;
    xr += xi * ri;
  }
  if (a.mode != 1) {
    __syncthreads();  // r of the CTA's range written
    const int N0 = a.pd.q * a.pd.P;
    const int b0 = coarse_block_of(a.pd, lo);
    const int b1 = hi >= a.pd.N ? N0 : coarse_block_of(a.pd, hi);
    const int l = threadIdx.x & (RL - 1);
    for (int bb = b0 + (int)threadIdx.x / RL; bb - (int)threadIdx.x / RL < b1;
         bb += FB_THREADS / RL) {
      double s = 0.0;
      const bool valid = bb < b1;
      if (valid) {
        int st, sz;
        coarse_block_range(a.pd, bb, st, sz);
        for (int k = l; k < sz; k += RL) s += a.r[st + k];
      }
      s += __shfl_xor_sync(0xffffffffu, s, 4);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      if (valid && l == 0) a.g0[bb] = s;
    }
  }
  double vv[2] = {rr, xr};
  reduce_finalize<2>(vv, a.ws, [&](double* t) {
    sc->rr = t[0];
    const double rel = sc->energy ? sqrt(fmax(-t[1], 0.0) / sc->esq0) : sqrt(t[0] / sc->bb);
    sc->rel = rel;
    sc->iter = iter + 1;
    if (!(rel == rel) || isinf(rel) || !(alpha == alpha) || isinf(alpha)) {
      sc->status = SFCDD_ERR_NAN;
      sc->done = 1;
    } else if (rel <= sc->rtol) {
      sc->done = 1;
    }
  });
}

template <int D>
int fused_blocks_d() {
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pcg_fused<D>, FB_THREADS, 0) !=
      cudaSuccess)
    return 0;
  return sms * std::min(occ, 2);
}

template <int D>
cudaError_t launch_fused_d(const FusedPcg& a, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)a.nblocks);
  cfg.blockDim = dim3(FB_THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_pcg_fused<D>, a);
}

}  // namespace

int fused_pcg_blocks(int d) {
  switch (d) {
    case 1: return fused_blocks_d<1>();
    case 2: return fused_blocks_d<2>();
    case 3: return fused_blocks_d<3>();
    case 4: return fused_blocks_d<4>();
    case 5: return fused_blocks_d<5>();
    case 6: return fused_blocks_d<6>();
    case 7: return fused_blocks_d<7>();
    default: return fused_blocks_d<8>();
  }
}

int launch_fused_pcg(const FusedPcg& a, cudaStream_t s) {
  cudaError_t e;
  switch (a.g.d) {
    case 1: e = launch_fused_d<1>(a, s); break;
    case 2: e = launch_fused_d<2>(a, s); break;
    case 3: e = launch_fused_d<3>(a, s); break;
    case 4: e = launch_fused_d<4>(a, s); break;
    case 5: e = launch_fused_d<5>(a, s); break;
    case 6: e = launch_fused_d<6>(a, s); break;
    case 7: e = launch_fused_d<7>(a, s); break;
    default: e = launch_fused_d<8>(a, s); break;
  }
  return e == cudaSuccess ? 0 : cuda_fail(e, "cooperative launch of k_pcg_fused", __FILE__, __LINE__);
}

}  // namespace sfcdd
