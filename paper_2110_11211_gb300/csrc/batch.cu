// Batched solve of many independent subgrid problems: the subproblems of the
// sparse-grid combination technique (Sec. 2: every level vector l of the
// layers |l|_1 = L + d - 1 - i gets its own anisotropic full grid, solved
// independently), each with its own number P_s of subdomains of the two-level
// SFC Schwarz method (eq. Pchoice: P = P_hat 2^{d-1-i} on layer i).
//
// One setup builds every subgrid into batch-wide arrays: a single radix sort of
// (subgrid, Hilbert key), per-subgrid descriptors, one tile-skyline set of all
// local matrices (FP64/FP32/BF16) and all coarse matrices (FP64).  The solve is
// one CUDA-graph launch whose conditional WHILE node repeats the PCG iteration
// of every subgrid until each has converged or maxit is reached: each subgrid
// has its own scalars and converged flag; converged subgrids skip their work.
// Per iteration: one kernel per subgrid CTA fuses stencil, p^T A p, the x/r
// update, the convergence test and the coarse restriction; the batched
// substitutions run all 24k+ local and coarse matrices; one kernel fuses the
// prolongation, r^T z, beta and the p update; one CTA sets the loop condition.
#include <algorithm>
#include <cstring>
#include <vector>

#include "device_common.cuh"

using namespace sfcdd;

namespace sfcdd {
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);
}

// One subgrid of the combination: vector offset, levels, lexicographic strides
// and the coefficient (-1)^i C(d-1, i) of its layer.
struct CombSub {
  int base;
  int lev[MAXD];
  int stride[MAXD];
  double coef;
};

struct sfcdd_batch {
  int nsub = 0, d = 0, precision = 0, weighting = 1, flexible = 0;
  double gamma = 0;
  Store st = Store::F64;
  cudaStream_t stream = nullptr, cap_stream = nullptr;
  std::vector<SubDesc> hsub;
  std::vector<long long> offs;  // nsub + 1 vector offsets
  SubDesc* dsub = nullptr;
  int Ntot = 0, maxN = 0, nlocal = 0, nmat = 0;
  unsigned* code = nullptr;
  int* invpad = nullptr;
  int *d_start = nullptr, *d_len = nullptr;
  double* d_omega = nullptr;
  int* d_msub = nullptr;  // subgrid of every local matrix
  CombSub* d_comb = nullptr;  // interpolation table of eq. combi (nsub)
  std::vector<CombSub> h_comb;
  std::vector<int> h_start;   // first curve position of every local matrix
  int nsub_local = 1, nsub_coarse = 1;
  TileSetDev ts{};
  int* d_nzr = nullptr;  // zero-row bounds (ts.nzr), written by the setup's scans
  MatDesc* d_md = nullptr;
  void* ltiles = nullptr;  // Lh tiles (unit diagonal blocks implied)
  void* lut = nullptr;     // Lh^T tiles, E_K on the diagonal
  double* ctiles = nullptr;
  double* cut = nullptr;
  SkylineHost sky;
  std::vector<int> h_nt, h_vbase;
  int max_nt_local = 0, max_nt_coarse = 0;
  TrsvWork *work_f = nullptr, *work_b = nullptr;
  int nwork = 0;
  unsigned long long *ticket_f = nullptr, *ticket_b = nullptr;
  // balanced operator (eq. balSW): local-only and coarse-only work lists, each
  // with its own ticket counters, and the vectors w = F r, r - A w, t
  int variant = SFCDD_ADDITIVE;
  struct List {
    TrsvWork *f = nullptr, *b = nullptr;
    int n = 0;
    unsigned long long *tf = nullptr, *tb = nullptr;
  } local_list, coarse_list;
  double *bw = nullptr, *bgg = nullptr, *bt = nullptr;
  double *ybuf = nullptr, *dbuf = nullptr, *zcbuf = nullptr;
  double *b = nullptr, *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr,
         *g0 = nullptr;
  PcgScalars* sc = nullptr;
  PcgScalars* sc_host = nullptr;
  ErrWord* err = nullptr;
  int* iter_counter = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_maxit = -1;
  double setup_ms = 0, solve_ms = 0;
  long long factor_bytes = 0;
  std::vector<void*> allocs;
};

namespace {

constexpr int BT = 512;  // threads of a per-subgrid CTA

template <class T>
int balloc(sfcdd_batch* b, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? SFCDD_ERR_NOMEM : SFCDD_ERR_CUDA;
  }
  b->allocs.push_back((void*)*p);
  return SFCDD_OK;
}

#define BTRY(x)                      \
  do {                               \
    int _rc = (x);                   \
    if (_rc != SFCDD_OK) return _rc; \
  } while (0)

void bfree(sfcdd_batch* b, void* p) {
  if (!p) return;
  for (auto& a : b->allocs)
    if (a == p) {
      cudaFree(p);
      a = nullptr;
    }
}

// Per-matrix substitution descriptors and the work lists of (matrix, tile row,
// slab) items for the given slab counts; drops the captured solve graph.
int batch_configure(sfcdd_batch* b, int nsub_local, int nsub_coarse) {
  cudaStream_t s = b->stream;
  if (nsub_local == 0 && !whole_fits(b->st, b->max_nt_local)) return SFCDD_ERR_INVALID_ARG;
  SFCDD_CUDA_OK(cudaStreamSynchronize(s));
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_maxit = -1;
  }
  b->nsub_local = nsub_local;
  b->nsub_coarse = nsub_coarse;
  std::vector<MatDesc> md(b->nmat);
  std::vector<int> nsl(b->nmat, nsub_local);
  for (int si = 0; si < b->nsub; ++si) {
    const SubDesc& sd = b->hsub[si];
    for (int i = 0; i < sd.pd.P; ++i)
      md[sd.mat0 + i] = {sd.base, sd.pd.N, b->h_start[(size_t)sd.mat0 + i], 0, si, nsub_local, 1};
    md[sd.cmat] = {sd.g0base, sd.N0, 0, 1, si, nsub_coarse, 1};
    nsl[sd.cmat] = nsub_coarse;
  }
  if (!b->d_md) BTRY(balloc(b, &b->d_md, b->nmat));
  SFCDD_CUDA_OK(cudaMemcpyAsync(b->d_md, md.data(), b->nmat * sizeof(MatDesc), cudaMemcpyHostToDevice, s));
  std::vector<TrsvWork> wf, wb;
  build_worklists(b->h_nt, std::vector<char>(b->nmat, 1), nsl, wf, wb);
  bfree(b, b->work_f);
  bfree(b, b->work_b);
  b->nwork = (int)wf.size();
  BTRY(balloc(b, &b->work_f, b->nwork));
  BTRY(balloc(b, &b->work_b, b->nwork));
  SFCDD_CUDA_OK(cudaMemcpyAsync(b->work_f, wf.data(), wf.size() * sizeof(TrsvWork), cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync(b->work_b, wb.data(), wb.size() * sizeof(TrsvWork), cudaMemcpyHostToDevice, s));
  if (!b->ticket_f) BTRY(balloc(b, &b->ticket_f, 1));
  if (!b->ticket_b) BTRY(balloc(b, &b->ticket_b, 1));
  SFCDD_CUDA_OK(cudaMemsetAsync(b->ticket_f, 0, sizeof(unsigned long long), s));
  SFCDD_CUDA_OK(cudaMemsetAsync(b->ticket_b, 0, sizeof(unsigned long long), s));
  if (b->variant == SFCDD_BALANCED) {
    for (int li = 0; li < 2; ++li) {
      std::vector<char> inc(b->nmat, li == 0 ? 1 : 0);
      for (int si = 0; si < b->nsub; ++si) inc[b->hsub[si].cmat] = li == 0 ? 0 : 1;
      std::vector<TrsvWork> lf, lb;
      build_worklists(b->h_nt, inc, nsl, lf, lb);
      auto& L = li == 0 ? b->local_list : b->coarse_list;
      bfree(b, L.f);
      bfree(b, L.b);
      L.n = (int)lf.size();
      BTRY(balloc(b, &L.f, L.n));
      BTRY(balloc(b, &L.b, L.n));
      SFCDD_CUDA_OK(cudaMemcpyAsync(L.f, lf.data(), lf.size() * sizeof(TrsvWork), cudaMemcpyHostToDevice, s));
      SFCDD_CUDA_OK(cudaMemcpyAsync(L.b, lb.data(), lb.size() * sizeof(TrsvWork), cudaMemcpyHostToDevice, s));
      if (!L.tf) BTRY(balloc(b, &L.tf, 1));
      if (!L.tb) BTRY(balloc(b, &L.tb, 1));
      SFCDD_CUDA_OK(cudaMemsetAsync(L.tf, 0, sizeof(unsigned long long), s));
      SFCDD_CUDA_OK(cudaMemsetAsync(L.tb, 0, sizeof(unsigned long long), s));
      SFCDD_CUDA_OK(cudaStreamSynchronize(s));
    }
  }
  SFCDD_CUDA_OK(cudaStreamSynchronize(s));  // host vectors go out of scope
  return SFCDD_OK;
}

// Deterministic block sum over BT threads; every thread gets the total.
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < BT / 32; ++k) t += sh[k];
  return t;
}

__device__ __forceinline__ int lex_id_of(const GridDev& g, unsigned c) {
  int id = 0;
  for (int j = 0; j < g.d; ++j) {
    const int kj = (int)((c >> g.off[j]) & ((1u << g.lev[j]) - 1u));
    id += (kj - 1) * g.stride[j];
  }
  return id;
}

// ---------------------------------------------------------------------------
// eq. combi: u_c(x) = sum_s c_s I_s u_s (x), I_s the piecewise multilinear
// interpolant of subgrid s's nodal values (zero Dirichlet data on the
// boundary nodes).  One warp per point; lane t sums the subgrids t, t + 32, ...
// in order and the warp adds the 32 partial sums in a fixed tree, so the result
// does not depend on timing.  Coordinates are clamped to [0, 1].  Corners on the
// boundary are skipped before their weight is formed (a level-1 axis has one
// interior node, so it halves the corners of its subgrid).
template <int D>
__global__ void __launch_bounds__(256) k_combine(const CombSub* __restrict__ cs, int nsub,
                                                 const double* __restrict__ u,
                                                 const double* __restrict__ pts, long long npts,
                                                 double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long p = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < npts;
       p += nwarps) {
    double x[D];
#pragma unroll
    for (int j = 0; j < D; ++j) x[j] = fmin(fmax(pts[p * D + j], 0.0), 1.0);
    double acc = 0.0;
    for (int t = lane; t < nsub; t += 32) {
      const CombSub& c = cs[t];
      int k[D];
      double fr[D];
      unsigned lo_out = 0u, hi_out = 0u;  // axes whose lower / upper node is a boundary node
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const int n = 1 << c.lev[j];
        const double tt = x[j] * (double)n;
        const int kk = min((int)floor(tt), n - 1);
        k[j] = kk;
        fr[j] = tt - (double)kk;
        if (kk == 0) lo_out |= 1u << j;
        if (kk + 1 == n) hi_out |= 1u << j;
      }
      double v = 0.0;
      for (unsigned corner = 0; corner < (1u << D); ++corner) {
        if ((~corner & lo_out) | (corner & hi_out)) continue;
        double w = 1.0;
        int id = 0;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          const int bit = (corner >> j) & 1;
          w *= bit ? fr[j] : 1.0 - fr[j];
          id += (k[j] + bit - 1) * c.stride[j];
        }
        v += w * u[(long long)c.base + id];
      }
      acc += c.coef * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) out[p] = acc;
  }
}

// ---------------------------------------------------------------------------
// Setup kernels.  grid.y = subgrid (or matrix), positions local to the subgrid.
template <int D>
__global__ void k_b_keygen(const SubDesc* __restrict__ sub, int kbits,
                           unsigned long long* __restrict__ keys, unsigned* __restrict__ codes) {
  const int s = blockIdx.y;
  const SubDesc& sd = sub[s];
  for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < sd.g.N; id += gridDim.x * blockDim.x) {
    unsigned c;
    const unsigned long long k = hilbert_key_of<D>(sd.g, id, c);
    keys[sd.base + id] = ((unsigned long long)s << kbits) | k;
    codes[sd.base + id] = c;
  }
}

__global__ void k_b_invpad(const SubDesc* __restrict__ sub, const unsigned* __restrict__ code,
                           int* __restrict__ invpad) {
  const SubDesc& sd = sub[blockIdx.y];
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < sd.g.N; p += gridDim.x * blockDim.x)
    invpad[sd.ibase + code[sd.base + p]] = p;
}

__global__ void k_b_env_local(const SubDesc* __restrict__ sub, const int* __restrict__ msub,
                              const unsigned* __restrict__ code, const int* __restrict__ invpad,
                              TileSetDev ts, int nlocal, int* tfirst) {
  const int m = grid_mat();
  if (m >= nlocal) return;
  const SubDesc& sd = sub[msub[m]];
  const int i = m - sd.mat0;
  const int n = ts.n[m];
  const int fb = ts.vbase[m] / TILE;
  const int start = sd.pd.start[i];
  const int vb = ts.vbase[m];
  const LocalOrder lo{ts.lperm ? ts.lperm + vb : nullptr, ts.linv ? ts.linv + vb : nullptr};
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const int first = envelope_row(sd.g, code + sd.base, invpad + sd.ibase, start, n, lo, r);
    if (first < r) atomicMin(&tfirst[fb + r / TILE], first);
  }
}

__global__ void k_b_env_coarse(const SubDesc* __restrict__ sub, const unsigned* __restrict__ code,
                               const int* __restrict__ invpad, TileSetDev ts, int* tfirst) {
  const SubDesc& sd = sub[blockIdx.y];
  const int fbc = ts.vbase[sd.cmat] / TILE;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < sd.g.N; p += gridDim.x * blockDim.x) {
    int a;
    const int first =
        envelope_coarse_point(sd.g, sd.pd, code + sd.base, invpad + sd.ibase, p, a);
    if (first < a) atomicMin(&tfirst[fbc + a / TILE], first);
  }
}

template <class T>
__device__ __forceinline__ T to_store(double v) { return T(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(double v) {
  return __float2bfloat16_rn((float)v);
}

template <class T>
__global__ void __launch_bounds__(256) k_b_assemble_local(const SubDesc* __restrict__ sub,
                                                          const int* __restrict__ msub,
                                                          const unsigned* __restrict__ code,
                                                          const int* __restrict__ invpad,
                                                          TileSetDev ts, int nlocal,
                                                          T* __restrict__ tiles) {
  __shared__ double sm[TILE2];
  const int m = grid_mat();
  if (m >= nlocal) return;
  const SubDesc& sd = sub[msub[m]];
  const int nt = ts.nt[m];
  const int fb = ts.vbase[m] / TILE;
  const int idx = blockIdx.x;
  if (idx >= stored_tiles(ts, fb, nt)) return;
  int a, bb;
  skyline_decode(ts, fb, nt, idx, a, bb);
  for (int k = threadIdx.x; k < TILE2; k += blockDim.x) sm[k] = 0.0;
  __syncthreads();
  const int vb = ts.vbase[m];
  const LocalOrder lo{ts.lperm ? ts.lperm + vb : nullptr, ts.linv ? ts.linv + vb : nullptr};
  assemble_local_tile(sd.g, code + sd.base, invpad + sd.ibase, sd.pd.start[m - sd.mat0], ts.n[m], lo, a,
                      bb, sm);
  __syncthreads();
  T* out = tiles + ts.tbase[m] + (long long)idx * TILE2;
  for (int k = threadIdx.x; k < TILE2; k += blockDim.x) out[k] = to_store<T>(sm[k]);
}

__global__ void __launch_bounds__(256) k_b_assemble_coarse(const SubDesc* __restrict__ sub,
                                                           const unsigned* __restrict__ code,
                                                           const int* __restrict__ invpad,
                                                           TileSetDev ts, double* __restrict__ tiles) {
  extern __shared__ __align__(16) unsigned char dsm_bc[];
  double* acc = reinterpret_cast<double*>(dsm_bc);
  int* cnt = reinterpret_cast<int*>(acc + TILE2);
  const SubDesc& sd = sub[blockIdx.y];
  const int m = sd.cmat;
  const int nt = ts.nt[m];
  const int fb = ts.vbase[m] / TILE;
  if ((int)blockIdx.x >= stored_tiles(ts, fb, nt)) return;
  int R, C;
  skyline_decode(ts, fb, nt, blockIdx.x, R, C);
  assemble_coarse_tile(sd.g, sd.pd, sd.N0, code + sd.base, invpad + sd.ibase, R, C, acc, cnt);
  double* out = tiles + ts.tbase[m] + (long long)blockIdx.x * TILE2;
  for (int k = threadIdx.x; k < TILE2; k += blockDim.x) out[k] = acc[k];
}

// ---------------------------------------------------------------------------
// Solve kernels: one CTA per subgrid.
__global__ void k_b_lex_to_curve(const SubDesc* __restrict__ sub, const unsigned* __restrict__ code,
                                 const double* __restrict__ in, double* __restrict__ out) {
  const SubDesc& sd = sub[blockIdx.y];
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < sd.g.N; p += gridDim.x * blockDim.x)
    out[sd.base + p] = in[sd.base + lex_id_of(sd.g, code[sd.base + p])];
}

__global__ void k_b_curve_to_lex(const SubDesc* __restrict__ sub, const unsigned* __restrict__ code,
                                 const double* __restrict__ in, double* __restrict__ out) {
  const SubDesc& sd = sub[blockIdx.y];
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < sd.g.N; p += gridDim.x * blockDim.x)
    out[sd.base + lex_id_of(sd.g, code[sd.base + p])] = in[sd.base + p];
}

__global__ void __launch_bounds__(BT) k_b_init(const SubDesc* __restrict__ sub,
                                               const double* __restrict__ b, double* __restrict__ x,
                                               double* __restrict__ r, double* __restrict__ p,
                                               double* __restrict__ z, PcgScalars* sc, double rtol,
                                               int flexible) {
  __shared__ double sh[BT / 32];
  const SubDesc& sd = sub[blockIdx.x];
  double acc = 0.0;
  for (int i = threadIdx.x; i < sd.g.N; i += BT) {
    const double bi = b[sd.base + i];
    x[sd.base + i] = 0.0;
    r[sd.base + i] = bi;
    p[sd.base + i] = 0.0;
    z[sd.base + i] = 0.0;
    acc += bi * bi;
  }
  const double bb = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    PcgScalars& c = sc[blockIdx.x];
    c.bb = bb;
    c.rr = bb;
    c.rel = bb > 0.0 ? 1.0 : 0.0;
    c.rz = c.rz_old = c.pq = c.alpha = c.beta = 0.0;
    c.iter = 0;
    c.status = 0;
    c.rtol = rtol;
    c.flexible = flexible;
    c.done = bb > 0.0 ? 0 : 1;
    if (!(bb == bb) || isinf(bb)) {  // non-finite right-hand side
      c.status = SFCDD_ERR_NAN;
      c.done = 1;
    }
  }
}

// g0 = R_0 r for one subgrid (eq. restr): warp per coarse block.
__device__ __forceinline__ void restrict_sub(const SubDesc& sd, const double* __restrict__ r,
                                             double* __restrict__ g0) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const PartDev& pd = sd.pd;
  for (int a = w; a < sd.N0; a += BT / 32) {
    const int t = a / pd.q, mm = a % pd.q;
    const int n = tilde_size(pd, t);
    const int bf = n / pd.q, br = n % pd.q;
    const int start = tilde_off(pd, t) + (mm < br ? mm * (bf + 1) : br * (bf + 1) + (mm - br) * bf);
    const int size = mm < br ? bf + 1 : bf;
    double s = 0.0;
    for (int k = lane; k < size; k += 32) s += r[sd.base + start + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) g0[sd.g0base + a] = s;
  }
}

__global__ void __launch_bounds__(BT) k_b_restrict(const SubDesc* __restrict__ sub,
                                                   const double* __restrict__ r,
                                                   double* __restrict__ g0, const PcgScalars* sc) {
  if (sc[blockIdx.x].done) return;
  restrict_sub(sub[blockIdx.x], r, g0);
}

// q = A p, alpha = r^T z / p^T q, x += alpha p, r -= alpha q, convergence test,
// then the coarse right-hand side R_0 r of the next preconditioner apply.
template <int D>
__global__ void __launch_bounds__(BT) k_b_iter(const SubDesc* __restrict__ sub,
                                               const unsigned* __restrict__ code,
                                               const int* __restrict__ invpad,
                                               const double* __restrict__ p, double* __restrict__ q,
                                               double* __restrict__ x, double* __restrict__ r,
                                               double* __restrict__ g0, PcgScalars* sc) {
  __shared__ double sh[BT / 32];
  PcgScalars& c = sc[blockIdx.x];
  if (c.done) return;
  const SubDesc& sd = sub[blockIdx.x];
  const unsigned* cs = code + sd.base;
  const int* ip = invpad + sd.ibase;
  const double* ps = p + sd.base;
  double acc = 0.0;
  for (int i = threadIdx.x; i < sd.g.N; i += BT) {
    double pi;
    const double v = stencil_point<D>(sd.g, cs, ip, ps, i, pi);
    q[sd.base + i] = v;
    acc += pi * v;
  }
  const double pq = block_sum(acc, sh);
  const double alpha = c.rz / pq;
  acc = 0.0;
  for (int i = threadIdx.x; i < sd.g.N; i += BT) {
    x[sd.base + i] += alpha * ps[i];
    const double ri = r[sd.base + i] - alpha * q[sd.base + i];
    r[sd.base + i] = ri;
    acc += ri * ri;
  }
  const double rr = block_sum(acc, sh);
  const double rel = sqrt(rr / c.bb);
  bool done = false;
  if (threadIdx.x == 0) {
    c.pq = pq;
    c.alpha = alpha;
    c.rr = rr;
    c.rel = rel;
    c.iter += 1;
    if (!(rel == rel) || isinf(rel) || !(alpha == alpha) || isinf(alpha)) {
      c.status = SFCDD_ERR_NAN;
      c.done = 1;
    } else if (rel <= c.rtol) {
      c.done = 1;
    }
  }
  done = !(rel == rel) || isinf(rel) || rel <= c.rtol;
  __syncthreads();
  if (!done) restrict_sub(sd, r, g0);
}

// z = R_0^T d_0 + sum_i omega_i R_i^T d_i, r^T z -> beta, p = z + beta p.
__global__ void __launch_bounds__(BT) k_b_prolong(const SubDesc* __restrict__ sub, TileSetDev ts,
                                                  const double* __restrict__ dvec,
                                                  const double* __restrict__ r,
                                                  double* __restrict__ z, double* __restrict__ p,
                                                  PcgScalars* sc) {
  __shared__ double sh[BT / 32];
  PcgScalars& c = sc[blockIdx.x];
  if (c.done) return;
  const SubDesc& sd = sub[blockIdx.x];
  const int cbase = ts.vbase[sd.cmat];
  auto lvbase = [&](int i) { return __ldg(&ts.vbase[sd.mat0 + i]); };
  double a1 = 0.0, a2 = 0.0;
  for (int i = threadIdx.x; i < sd.g.N; i += BT) {
    const double v = prolong_point(sd.pd, 0, dvec, cbase, lvbase, ts.linv, i);
    const double ri = r[sd.base + i];
    a1 += ri * v;
    a2 += ri * z[sd.base + i];
    z[sd.base + i] = v;
  }
  const double rz_new = block_sum(a1, sh);
  const double rz_old = block_sum(a2, sh);
  double beta;
  if (c.iter == 0) beta = 0.0;
  else if (c.flexible) beta = (rz_new - rz_old) / c.rz;
  else beta = rz_new / c.rz;
  __syncthreads();
  if (threadIdx.x == 0) {
    c.beta = beta;
    c.rz_old = rz_old;
    c.rz = rz_new;
  }
  for (int i = threadIdx.x; i < sd.g.N; i += BT) p[sd.base + i] = z[sd.base + i] + beta * p[sd.base + i];
}


// Balanced operator (eq. balSW), z = t - F A t + w with w = F r and
// t = C_(1) (r - A w), in three per-subgrid kernels between substitution pairs
// over the coarse-only and the local-only work lists.  Each CTA owns its whole
// subgrid, so a vector it writes is complete for its stencil after a barrier.
// 1: w = R_0^T d_0 (from the coarse solve of R_0 r), gg = r - A w.
template <int D>
__global__ void __launch_bounds__(BT) k_b_bal_w(const SubDesc* __restrict__ sub,
                                                const unsigned* __restrict__ code,
                                                const int* __restrict__ invpad, TileSetDev ts,
                                                const double* __restrict__ dvec,
                                                const double* __restrict__ r, double* __restrict__ w,
                                                double* __restrict__ gg, const PcgScalars* sc) {
  if (sc[blockIdx.x].done) return;
  const SubDesc& sd = sub[blockIdx.x];
  const int cbase = ts.vbase[sd.cmat];
  auto lvbase = [&](int i) { return __ldg(&ts.vbase[sd.mat0 + i]); };
  for (int i = threadIdx.x; i < sd.g.N; i += BT)
    w[sd.base + i] = prolong_point(sd.pd, 2, dvec, cbase, lvbase, ts.linv, i);
  __syncthreads();
  for (int i = threadIdx.x; i < sd.g.N; i += BT) {
    double wi;
    const double aw = stencil_point<D>(sd.g, code + sd.base, invpad + sd.ibase, w + sd.base, i, wi);
    gg[sd.base + i] = r[sd.base + i] - aw;
  }
}

// 2: t = sum_i omega_i R_i^T d_i (local solves of gg), g0 = R_0 A t (A t in q).
template <int D>
__global__ void __launch_bounds__(BT) k_b_bal_t(const SubDesc* __restrict__ sub,
                                                const unsigned* __restrict__ code,
                                                const int* __restrict__ invpad, TileSetDev ts,
                                                const double* __restrict__ dvec,
                                                double* __restrict__ t, double* __restrict__ q,
                                                double* __restrict__ g0, const PcgScalars* sc) {
  if (sc[blockIdx.x].done) return;
  const SubDesc& sd = sub[blockIdx.x];
  const int cbase = ts.vbase[sd.cmat];
  auto lvbase = [&](int i) { return __ldg(&ts.vbase[sd.mat0 + i]); };
  for (int i = threadIdx.x; i < sd.g.N; i += BT)
    t[sd.base + i] = prolong_point(sd.pd, 1, dvec, cbase, lvbase, ts.linv, i);
  __syncthreads();
  for (int i = threadIdx.x; i < sd.g.N; i += BT) {
    double ti;
    q[sd.base + i] = stencil_point<D>(sd.g, code + sd.base, invpad + sd.ibase, t + sd.base, i, ti);
  }
  __syncthreads();
  restrict_sub(sd, q, g0);
}

// 3: v = R_0^T d_0 (coarse solve of R_0 A t), z = t - v + w, r^T z -> beta,
// p = z + beta p.
__global__ void __launch_bounds__(BT) k_b_bal_z(const SubDesc* __restrict__ sub, TileSetDev ts,
                                                const double* __restrict__ dvec,
                                                const double* __restrict__ t,
                                                const double* __restrict__ w,
                                                const double* __restrict__ r,
                                                double* __restrict__ z, double* __restrict__ p,
                                                PcgScalars* sc) {
  __shared__ double sh[BT / 32];
  PcgScalars& c = sc[blockIdx.x];
  if (c.done) return;
  const SubDesc& sd = sub[blockIdx.x];
  const int cbase = ts.vbase[sd.cmat];
  auto lvbase = [&](int i) { return __ldg(&ts.vbase[sd.mat0 + i]); };
  double a1 = 0.0, a2 = 0.0;
  for (int i = threadIdx.x; i < sd.g.N; i += BT) {
    const double v = prolong_point(sd.pd, 2, dvec, cbase, lvbase, ts.linv, i);
    const double zi = t[sd.base + i] - v + w[sd.base + i];
    const double ri = r[sd.base + i];
    a1 += ri * zi;
    a2 += ri * z[sd.base + i];
    z[sd.base + i] = zi;
  }
  const double rz_new = block_sum(a1, sh);
  const double rz_old = block_sum(a2, sh);
  double beta;
  if (c.iter == 0) beta = 0.0;
  else if (c.flexible) beta = (rz_new - rz_old) / c.rz;
  else beta = rz_new / c.rz;
  __syncthreads();
  if (threadIdx.x == 0) {
    c.beta = beta;
    c.rz_old = rz_old;
    c.rz = rz_new;
  }
  for (int i = threadIdx.x; i < sd.g.N; i += BT) p[sd.base + i] = z[sd.base + i] + beta * p[sd.base + i];
}

// Loop condition of the graph's WHILE node: another iteration while any
// subgrid is still running and fewer than maxit iterations have been done.
__global__ void k_b_cond(const PcgScalars* sc, int nsub, int* iter_counter, int maxit,
                         cudaGraphConditionalHandle cond) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  int mine = 0;
  for (int s = threadIdx.x; s < nsub; s += blockDim.x) mine |= (sc[s].done == 0);
  if (mine) atomicOr(&any, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int it = *iter_counter + 1;
    *iter_counter = it;
    cudaGraphSetConditional(cond, (any && it < maxit) ? 1u : 0u);
  }
}

template <int D>
__global__ void __launch_bounds__(BT) k_b_true_res(const SubDesc* __restrict__ sub,
                                                   const unsigned* __restrict__ code,
                                                   const int* __restrict__ invpad,
                                                   const double* __restrict__ b,
                                                   const double* __restrict__ x, PcgScalars* sc) {
  __shared__ double sh[BT / 32];
  const SubDesc& sd = sub[blockIdx.x];
  double acc = 0.0;
  for (int i = threadIdx.x; i < sd.g.N; i += BT) {
    double xi;
    const double v = b[sd.base + i] -
                     stencil_point<D>(sd.g, code + sd.base, invpad + sd.ibase, x + sd.base, i, xi);
    acc += v * v;
  }
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) sc[blockIdx.x].true_rel = sc[blockIdx.x].bb > 0 ? sqrt(t / sc[blockIdx.x].bb) : 0.0;
}

#define SFCDD_DISPATCH_D(KERNEL, d, grid, block, smem, stream, ...)                 \
  switch (d) {                                                                      \
    case 1: KERNEL<1><<<grid, block, smem, stream>>>(__VA_ARGS__); break;           \
    case 2: KERNEL<2><<<grid, block, smem, stream>>>(__VA_ARGS__); break;           \
    case 3: KERNEL<3><<<grid, block, smem, stream>>>(__VA_ARGS__); break;           \
    case 4: KERNEL<4><<<grid, block, smem, stream>>>(__VA_ARGS__); break;           \
    case 5: KERNEL<5><<<grid, block, smem, stream>>>(__VA_ARGS__); break;           \
    case 6: KERNEL<6><<<grid, block, smem, stream>>>(__VA_ARGS__); break;           \
    case 7: KERNEL<7><<<grid, block, smem, stream>>>(__VA_ARGS__); break;           \
    default: KERNEL<8><<<grid, block, smem, stream>>>(__VA_ARGS__); break;          \
  }

// list 0: every matrix; 1: the local matrices; 2: the coarse matrices
TrsvArgs batch_trsv_args(sfcdd_batch* b, bool fwd, int list = 0, const double* rhs = nullptr) {
  TrsvArgs a{};
  a.ts = b->ts;
  a.md = b->d_md;
  a.ltiles = b->ltiles;
  a.lut = b->lut;
  a.ctiles = b->ctiles;
  a.cut = b->cut;
  a.zc = b->zcbuf;
  a.rhs = b->r;
  a.g0 = b->g0;
  a.y = b->ybuf;
  a.dout = b->dbuf;
  a.work = fwd ? b->work_f : b->work_b;
  a.nwork = b->nwork;
  a.ticket = fwd ? b->ticket_f : b->ticket_b;
  if (list != 0) {
    const auto& L = list == 1 ? b->local_list : b->coarse_list;
    a.work = fwd ? L.f : L.b;
    a.nwork = L.n;
    a.ticket = fwd ? L.tf : L.tb;
  }
  if (rhs) a.rhs = rhs;
  a.err = b->err;
  a.sc = b->sc;
  if (b->nsub_local == 0 && list != 2) a.zv_doubles = b->max_nt_local * TILE;
  return a;
}

void enqueue_pair(sfcdd_batch* b, int list, const double* rhs, cudaStream_t s) {
  launch_trsv_fwd(batch_trsv_args(b, true, list, rhs), b->st, s);
  launch_trsv_bwd(batch_trsv_args(b, false, list, rhs), b->st, s);
}

// z = C^{-1} r for every subgrid (R_0 r already in g0), r^T z, beta, p update
void enqueue_apply(sfcdd_batch* b, cudaStream_t s) {
  if (b->variant != SFCDD_BALANCED) {
    enqueue_pair(b, 0, nullptr, s);
    k_b_prolong<<<b->nsub, BT, 0, s>>>(b->dsub, b->ts, b->dbuf, b->r, b->z, b->p, b->sc);
    return;
  }
  enqueue_pair(b, 2, nullptr, s);  // d_0 = A_0^{-1} R_0 r
  SFCDD_DISPATCH_D(k_b_bal_w, b->d, b->nsub, BT, 0, s, b->dsub, b->code, b->invpad, b->ts, b->dbuf,
                   b->r, b->bw, b->bgg, b->sc);
  enqueue_pair(b, 1, b->bgg, s);   // d_i = A_i^{-1} R_i (r - A w)
  SFCDD_DISPATCH_D(k_b_bal_t, b->d, b->nsub, BT, 0, s, b->dsub, b->code, b->invpad, b->ts, b->dbuf,
                   b->bt, b->q, b->g0, b->sc);
  enqueue_pair(b, 2, nullptr, s);  // d_0 = A_0^{-1} R_0 A t
  k_b_bal_z<<<b->nsub, BT, 0, s>>>(b->dsub, b->ts, b->dbuf, b->bt, b->bw, b->r, b->z, b->p, b->sc);
}

int build_graph(sfcdd_batch* b, int maxit) {
  if (b->graph && b->graph_maxit == maxit) return SFCDD_OK;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaGraph_t graph;
  SFCDD_CUDA_OK(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle cond;
  SFCDD_CUDA_OK(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  SFCDD_CUDA_OK(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaStream_t cs = b->cap_stream;
  SFCDD_CUDA_OK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal));
  SFCDD_DISPATCH_D(k_b_iter, b->d, b->nsub, BT, 0, cs, b->dsub, b->code, b->invpad, b->p, b->q,
                   b->x, b->r, b->g0, b->sc);
  enqueue_apply(b, cs);
  k_b_cond<<<1, 256, 0, cs>>>(b->sc, b->nsub, b->iter_counter, maxit, cond);
  cudaGraph_t captured;
  cudaError_t e = cudaStreamEndCapture(cs, &captured);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
  }
  e = cudaGraphInstantiate(&b->graph, graph, 0);
  cudaGraphDestroy(graph);
  SFCDD_CUDA_OK(e);
  b->graph_maxit = maxit;
  return SFCDD_OK;
}

int batch_setup_impl(sfcdd_batch* b, const int* levels, int nsub, int d, const int* Ps,
                     double overlap, const sfcdd_options* opt) {
  NvtxRange nvtx("sfcdd batch setup");
  if (!levels || !Ps || nsub < 1 || d < 1 || d > MAXD || !(overlap > 0))
    return SFCDD_ERR_INVALID_ARG;
  if (nsub > 65535) return SFCDD_ERR_UNSUPPORTED;  // per-subgrid launches index grid.y
  for (int si = 0; si < nsub; ++si)
    if (Ps[si] < 2) return SFCDD_ERR_INVALID_ARG;
  sfcdd_options o;
  sfcdd_default_options(&o);
  if (opt) o = *opt;
  const bool variant_ok = o.variant == SFCDD_ADDITIVE || o.variant == SFCDD_BALANCED;
  if (!variant_ok || o.precision < 0 || o.precision > 2 || o.weighting < 0 || o.weighting > 1 ||
      o.tensor_cores < -1 || o.tensor_cores > 2)
    return !variant_ok ? SFCDD_ERR_UNSUPPORTED : SFCDD_ERR_INVALID_ARG;
  b->variant = o.variant;
  b->nsub = nsub;
  b->d = d;
  b->gamma = overlap;
  b->precision = o.precision;
  b->weighting = o.weighting;
  b->flexible = o.flexible < 0 ? (o.precision != SFCDD_FP64 ? 1 : 0) : (o.flexible ? 1 : 0);
  b->st = (Store)o.precision;
  b->stream = (cudaStream_t)o.stream;
  cudaStream_t s = b->stream;
  SFCDD_CUDA_OK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  SFCDD_CUDA_OK(cudaEventCreate(&e0));
  SFCDD_CUDA_OK(cudaEventCreate(&e1));
  SFCDD_CUDA_OK(cudaEventRecord(e0, s));

  // per-subgrid grids and partitions (host)
  b->hsub.resize(nsub);
  b->offs.assign(nsub + 1, 0);
  std::vector<int> start_all, len_all;
  std::vector<double> omega_all;
  std::vector<int> N0s(nsub);
  long long ibase = 0, base = 0;
  int kbits = 0;
  std::vector<int> pofs(nsub + 1, 0);  // first local matrix of every subgrid
  for (int si = 0; si < nsub; ++si) {
    SubDesc& sd = b->hsub[si];
    const int P = Ps[si];
    long long N;
    int B;
    BTRY(make_grid(levels + (size_t)si * d, d, o.coeffs, sd.g, N, B));
    if (P > N) return SFCDD_ERR_INVALID_ARG;
    pofs[si + 1] = pofs[si] + P;
    std::vector<int> st, ln;
    std::vector<double> om;
    int gf;
    BTRY(partition_ranges(N, P, overlap, o.weighting, st, ln, om, gf));
    const int q = o.q <= 0 ? paper_q(N, P) : o.q;
    if (q < 1 || q > N / P) return SFCDD_ERR_INVALID_ARG;
    sd.pd.N = (int)N;
    sd.pd.P = P;
    sd.pd.q = q;
    sd.pd.g = gf;
    sd.pd.f = (int)(N / P);
    sd.pd.r = (int)(N % P);
    sd.base = (int)base;
    sd.ibase = (int)ibase;
    sd.N0 = q * P;
    N0s[si] = sd.N0;
    start_all.insert(start_all.end(), st.begin(), st.end());
    len_all.insert(len_all.end(), ln.begin(), ln.end());
    omega_all.insert(omega_all.end(), om.begin(), om.end());
    b->offs[si] = base;
    base += N;
    ibase += 1ll << B;
    kbits = std::max(kbits, d * sd.g.nbits);
    b->maxN = std::max(b->maxN, (int)N);
  }
  b->offs[nsub] = base;
  if (base >= (1ll << 31) || ibase >= (1ll << 31)) return SFCDD_ERR_UNSUPPORTED;
  int sbits = 0;
  while ((1 << sbits) < nsub) ++sbits;
  if (kbits + sbits > 64) return SFCDD_ERR_KEY_OVERFLOW;
  b->Ntot = (int)base;
  b->nlocal = pofs[nsub];
  BTRY(balloc(b, &b->d_start, b->nlocal));
  BTRY(balloc(b, &b->d_len, b->nlocal));
  BTRY(balloc(b, &b->d_omega, b->nlocal));
  SFCDD_CUDA_OK(cudaMemcpyAsync(b->d_start, start_all.data(), start_all.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync(b->d_len, len_all.data(), len_all.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync(b->d_omega, omega_all.data(), omega_all.size() * sizeof(double), cudaMemcpyHostToDevice, s));

  // matrices: locals pofs[s] + i, coarse nlocal + s
  std::vector<int> hmsub(b->nlocal);
  for (int si = 0; si < nsub; ++si)
    for (int m = pofs[si]; m < pofs[si + 1]; ++m) hmsub[m] = si;
  BTRY(balloc(b, &b->d_msub, b->nlocal));
  SFCDD_CUDA_OK(cudaMemcpyAsync(b->d_msub, hmsub.data(), b->nlocal * sizeof(int), cudaMemcpyHostToDevice, s));
  b->nmat = b->nlocal + nsub;
  std::vector<int> h_n(b->nmat);
  b->h_nt.assign(b->nmat, 0);
  b->h_vbase.assign(b->nmat, 0);
  std::vector<char> is_coarse(b->nmat, 0);
  long long vb = 0;
  for (int m = 0; m < b->nmat; ++m) {
    int n;
    if (m < b->nlocal) {
      n = len_all[m];
    } else {
      n = N0s[m - b->nlocal];
      is_coarse[m] = 1;
    }
    h_n[m] = n;
    b->h_nt[m] = (n + TILE - 1) / TILE;
    b->h_vbase[m] = (int)vb;
    vb += (long long)b->h_nt[m] * TILE;
    if (m < b->nlocal) b->max_nt_local = std::max(b->max_nt_local, b->h_nt[m]);
    else b->max_nt_coarse = std::max(b->max_nt_coarse, b->h_nt[m]);
  }
  if (vb >= (1ll << 31)) return SFCDD_ERR_UNSUPPORTED;
  const int nrows = (int)(vb / TILE);
  long long g0base = 0;
  for (int si = 0; si < nsub; ++si) {
    SubDesc& sd = b->hsub[si];
    sd.pd.start = b->d_start + pofs[si];
    sd.pd.len = b->d_len + pofs[si];
    sd.pd.omega = b->d_omega + pofs[si];
    sd.mat0 = pofs[si];
    sd.cmat = b->nlocal + si;
    sd.g0base = (int)g0base;
    g0base += (long long)b->h_nt[sd.cmat] * TILE;
  }
  BTRY(balloc(b, &b->dsub, nsub));
  SFCDD_CUDA_OK(cudaMemcpyAsync(b->dsub, b->hsub.data(), nsub * sizeof(SubDesc), cudaMemcpyHostToDevice, s));
  BTRY(balloc(b, &b->d_comb, nsub));
  b->h_comb.assign(nsub, CombSub{});
  for (int si = 0; si < nsub; ++si) {
    CombSub& c = b->h_comb[si];
    c.base = b->hsub[si].base;
    for (int j = 0; j < MAXD; ++j) {
      c.lev[j] = j < d ? b->hsub[si].g.lev[j] : 0;
      c.stride[j] = j < d ? b->hsub[si].g.stride[j] : 0;
    }
  }

  // curve order of every subgrid: one sort of (subgrid, key)
  unsigned long long* keys;
  unsigned char* sort_tmp;
  BTRY(balloc(b, &keys, b->Ntot));
  BTRY(balloc(b, &b->code, b->Ntot));
  BTRY(balloc(b, &sort_tmp, radix_sort_temp_bytes(b->Ntot)));
  BTRY(balloc(b, &b->invpad, ibase));
  const dim3 gsub((b->maxN + 255) / 256, nsub);
  SFCDD_DISPATCH_D(k_b_keygen, d, gsub, 256, 0, s, b->dsub, kbits, keys, b->code);
  radix_sort_pairs(keys, b->code, b->Ntot, kbits + sbits, sort_tmp, s, nullptr);
  SFCDD_CUDA_OK(cudaMemsetAsync(b->invpad, 0xff, ibase * sizeof(int), s));
  k_b_invpad<<<gsub, 256, 0, s>>>(b->dsub, b->code, b->invpad);
  SFCDD_CUDA_OK(cudaGetLastError());

  // tile layout, local numbering (lexicographic by default) and envelopes
  int *d_n, *d_nt, *d_vbase, *tfirst;
  long long* d_tbase;
  BTRY(balloc(b, &d_n, b->nmat));
  BTRY(balloc(b, &d_nt, b->nmat));
  BTRY(balloc(b, &d_vbase, b->nmat));
  BTRY(balloc(b, &d_tbase, b->nmat));
  BTRY(balloc(b, &tfirst, nrows));
  SFCDD_CUDA_OK(cudaMemcpyAsync(d_n, h_n.data(), b->nmat * sizeof(int), cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync(d_nt, b->h_nt.data(), b->nmat * sizeof(int), cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync(d_vbase, b->h_vbase.data(), b->nmat * sizeof(int), cudaMemcpyHostToDevice, s));
  b->ts.nmat = b->nmat;
  b->ts.n = d_n;
  b->ts.nt = d_nt;
  b->ts.vbase = d_vbase;
  b->ts.tbase = d_tbase;
  const int max_nt_all = std::max(b->max_nt_local, b->max_nt_coarse);
  int max_nl = 0;
  for (int m = 0; m < b->nlocal; ++m) max_nl = std::max(max_nl, h_n[m]);
  if (o.local_order == 0) {
    std::vector<int> mstart(b->nlocal), mN(b->nlocal), mcb(b->nlocal), lb(b->nlocal);
    long long tot = 0;
    for (int m = 0; m < b->nlocal; ++m) {
      const SubDesc& sd = b->hsub[hmsub[m]];
      mstart[m] = start_all[m];
      mN[m] = sd.pd.N;
      mcb[m] = sd.base;
      lb[m] = (int)tot;
      tot += h_n[m];
    }
    int *d_ms, *d_mN, *d_mcb, *d_lb, *lperm, *linv;
    unsigned long long* okeys;
    unsigned* ovals;
    unsigned char* otemp;
    BTRY(balloc(b, &d_ms, b->nlocal));
    BTRY(balloc(b, &d_mN, b->nlocal));
    BTRY(balloc(b, &d_mcb, b->nlocal));
    BTRY(balloc(b, &d_lb, b->nlocal));
    BTRY(balloc(b, &lperm, vb));
    BTRY(balloc(b, &linv, vb));
    BTRY(balloc(b, &okeys, tot));
    BTRY(balloc(b, &ovals, tot));
    BTRY(balloc(b, &otemp, radix_sort_temp_bytes((int)tot)));
    SFCDD_CUDA_OK(cudaMemcpyAsync(d_ms, mstart.data(), b->nlocal * sizeof(int), cudaMemcpyHostToDevice, s));
    SFCDD_CUDA_OK(cudaMemcpyAsync(d_mN, mN.data(), b->nlocal * sizeof(int), cudaMemcpyHostToDevice, s));
    SFCDD_CUDA_OK(cudaMemcpyAsync(d_mcb, mcb.data(), b->nlocal * sizeof(int), cudaMemcpyHostToDevice, s));
    SFCDD_CUDA_OK(cudaMemcpyAsync(d_lb, lb.data(), b->nlocal * sizeof(int), cudaMemcpyHostToDevice, s));
    local_order_lex(b->ts, b->nlocal, max_nl, d_ms, d_mN, d_mcb, d_lb, tot, b->code, okeys, ovals,
                    otemp, lperm, linv, s);
    SFCDD_CUDA_OK(cudaStreamSynchronize(s));
    for (auto& a : b->allocs)
      if (a == okeys || a == ovals || a == otemp) {
        cudaFree(a);
        a = nullptr;
      }
    b->ts.lperm = lperm;
    b->ts.linv = linv;
  }
  launch_envelope_init(b->ts, b->nmat, max_nt_all, tfirst, s);
  k_b_env_local<<<mat_grid((max_nl + 255) / 256, b->nlocal), 256, 0, s>>>(
      b->dsub, b->d_msub, b->code, b->invpad, b->ts, b->nlocal, tfirst);
  k_b_env_coarse<<<gsub, 256, 0, s>>>(b->dsub, b->code, b->invpad, b->ts, tfirst);
  std::vector<int> tf(nrows);
  SFCDD_CUDA_OK(cudaMemcpyAsync(tf.data(), tfirst, nrows * sizeof(int), cudaMemcpyDeviceToHost, s));
  SFCDD_CUDA_OK(cudaStreamSynchronize(s));
  build_skyline(b->h_nt, b->h_vbase, is_coarse, std::vector<int>(b->nmat, 1), tf, b->sky);
  int *d_kmin, *d_rowoff, *d_colptr, *d_colidx;
  BTRY(balloc(b, &d_kmin, nrows));
  BTRY(balloc(b, &d_rowoff, nrows));
  BTRY(balloc(b, &d_colptr, nrows + 1));
  BTRY(balloc(b, &d_colidx, b->sky.colidx.size()));
  SFCDD_CUDA_OK(cudaMemcpyAsync(d_kmin, b->sky.kmin.data(), nrows * sizeof(int), cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync(d_rowoff, b->sky.rowoff.data(), nrows * sizeof(int), cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync(d_colptr, b->sky.colptr.data(), (nrows + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync(d_colidx, b->sky.colidx.data(), b->sky.colidx.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync(d_tbase, b->sky.tbase.data(), b->nmat * sizeof(long long), cudaMemcpyHostToDevice, s));
  b->ts.kmin = d_kmin;
  b->ts.rowoff = d_rowoff;
  b->ts.colptr = d_colptr;
  b->ts.colidx = d_colidx;
  // zero-row bounds of the off-block tiles: whole tiles until the factors are scanned
  {
    BTRY(balloc(b, &b->d_nzr, nrows));
    const std::vector<int> whole(nrows, TILE);
    SFCDD_CUDA_OK(cudaMemcpyAsync(b->d_nzr, whole.data(), nrows * sizeof(int), cudaMemcpyHostToDevice, s));
    SFCDD_CUDA_OK(cudaStreamSynchronize(s));
    b->ts.nzr = b->d_nzr;
  }

  // local matrices and factors (Sec. 3.1), coarse matrices and FP64 factors (eq. csm)
  BTRY(balloc(b, &b->err, 1));
  SFCDD_CUDA_OK(cudaMemsetAsync(b->err, 0, sizeof(ErrWord), s));
  int* diag_cnt = nullptr;  // per tile row: updates of its diagonal tile seen (factorization)
  BTRY(balloc(b, &diag_cnt, nrows));
  SFCDD_CUDA_OK(cudaMemsetAsync(diag_cnt, 0, nrows * sizeof(int), s));
  const Store cst = b->st == Store::BF16 ? Store::F32 : b->st;
  const size_t esz = cst == Store::F64 ? 8 : 4;
  void* work_tiles = nullptr;
  BTRY(balloc(b, (unsigned char**)&work_tiles, b->sky.ltiles * TILE2 * esz));
  switch (cst) {
    case Store::F64:
      k_b_assemble_local<double><<<mat_grid(b->sky.max_ltiles, b->nlocal), 256, 0, s>>>(
          b->dsub, b->d_msub, b->code, b->invpad, b->ts, b->nlocal, (double*)work_tiles);
      break;
    default:
      k_b_assemble_local<float><<<mat_grid(b->sky.max_ltiles, b->nlocal), 256, 0, s>>>(
          b->dsub, b->d_msub, b->code, b->invpad, b->ts, b->nlocal, (float*)work_tiles);
      break;
  }
  struct NoHook : LaunchHook {
    void before(int) override {}
    void after(int) override {}
  } nohook;
  factor_tiles(b->ts, 0, b->nlocal, b->max_nt_local, b->sky.col_max_local.data(), work_tiles, cst,
               diag_cnt, b->err, s, &nohook, 1, o.tensor_cores != 0,
               o.precision == SFCDD_BF16 && o.tensor_cores != 0 && o.tensor_cores != 2);
  // substitution form: Lh in place, Lh^T and E_K into a second tile array
  void* work_ut = nullptr;
  BTRY(balloc(b, (unsigned char**)&work_ut, b->sky.ltiles * TILE2 * esz));
  unitize_tiles(b->ts, 0, b->nlocal, b->sky.max_ltiles, work_tiles, work_ut, cst, s);
  if (b->st == Store::BF16) {
    BTRY(balloc(b, (__nv_bfloat16**)&b->ltiles, b->sky.ltiles * TILE2));
    BTRY(balloc(b, (__nv_bfloat16**)&b->lut, b->sky.ltiles * TILE2));
    launch_convert_f32_bf16((const float*)work_tiles, (__nv_bfloat16*)b->ltiles, b->sky.ltiles * TILE2, s);
    launch_convert_f32_bf16((const float*)work_ut, (__nv_bfloat16*)b->lut, b->sky.ltiles * TILE2, s);
    SFCDD_CUDA_OK(cudaStreamSynchronize(s));
    cudaFree(work_tiles);
    cudaFree(work_ut);
    for (auto& a : b->allocs)
      if (a == work_tiles || a == work_ut) a = nullptr;
  } else {
    b->ltiles = work_tiles;
    b->lut = work_ut;
  }
  launch_offblock_rows(b->ts, 0, b->nlocal, b->max_nt_local, b->ltiles, b->st,
                       b->d_nzr, s);
  if (b->st == Store::F64)
    launch_pack_half_tiles(b->ts, 0, b->nlocal, b->sky.max_ltiles, (double*)b->lut, b->d_nzr, s);
  BTRY(balloc(b, &b->ctiles, b->sky.ctiles * TILE2));
  {
    const int smem = TILE2 * (int)(sizeof(double) + sizeof(int));
    cudaFuncSetAttribute(k_b_assemble_coarse, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_b_assemble_coarse<<<dim3(b->sky.max_ctiles, nsub), 256, smem, s>>>(b->dsub, b->code, b->invpad,
                                                                        b->ts, b->ctiles);
  }
  factor_tiles(b->ts, b->nlocal, nsub, b->max_nt_coarse, b->sky.col_max_coarse.data(), b->ctiles,
               Store::F64, diag_cnt, b->err, s, &nohook, 1, o.tensor_cores != 0);
  BTRY(balloc(b, &b->cut, b->sky.ctiles * TILE2));
  unitize_tiles(b->ts, b->nlocal, nsub, b->sky.max_ctiles, b->ctiles, b->cut, Store::F64, s);
  launch_offblock_rows(b->ts, b->nlocal, nsub, b->max_nt_coarse, b->ctiles, Store::F64,
                       b->d_nzr, s);
  launch_pack_half_tiles(b->ts, b->nlocal, nsub, b->sky.max_ctiles, b->cut, b->d_nzr, s);
  SFCDD_CUDA_OK(cudaGetLastError());
  b->factor_bytes = b->sky.ltiles * TILE2 * (b->precision == 0 ? 8 : b->precision == 1 ? 4 : 2) +
                    b->sky.ctiles * TILE2 * 8;

  // substitution descriptors and work lists (FP32 / BF16 launches run the FP64
  // coarse rows in 16-row slabs; sfcdd_batch_autotune may change both counts)
  b->h_start = start_all;
  {
    // slabs_local -1: one CTA per local matrix (internal 0)
    const int sl = o.slabs_local == 0 ? 1 : (o.slabs_local == -1 ? 0 : o.slabs_local);
    const int sc = o.slabs_coarse == 0 ? (b->st == Store::F64 ? 1 : 4) : o.slabs_coarse;
    const bool ok = (sl == 0 || sl == 1 || sl == 2 || sl == 4) && (sc == 1 || sc == 2 || sc == 4) &&
                    (b->st == Store::F64 || sc != 1);
    if (!ok) return SFCDD_ERR_INVALID_ARG;
    BTRY(batch_configure(b, sl, sc));
  }
  BTRY(balloc(b, &b->ybuf, vb));
  BTRY(balloc(b, &b->dbuf, vb));
  BTRY(balloc(b, &b->zcbuf, vb));
  launch_fill_pending(b->ybuf, vb, s);
  launch_fill_pending(b->dbuf, vb, s);

  // PCG state
  BTRY(balloc(b, &b->b, b->Ntot));
  BTRY(balloc(b, &b->x, b->Ntot));
  BTRY(balloc(b, &b->r, b->Ntot));
  BTRY(balloc(b, &b->p, b->Ntot));
  BTRY(balloc(b, &b->q, b->Ntot));
  BTRY(balloc(b, &b->z, b->Ntot));
  if (b->variant == SFCDD_BALANCED) {
    BTRY(balloc(b, &b->bw, b->Ntot));
    BTRY(balloc(b, &b->bgg, b->Ntot));
    BTRY(balloc(b, &b->bt, b->Ntot));
  }
  BTRY(balloc(b, &b->g0, std::max<long long>(g0base, 1)));
  SFCDD_CUDA_OK(cudaMemsetAsync(b->g0, 0, std::max<long long>(g0base, 1) * sizeof(double), s));
  BTRY(balloc(b, &b->sc, nsub));
  SFCDD_CUDA_OK(cudaMemsetAsync(b->sc, 0, nsub * sizeof(PcgScalars), s));
  SFCDD_CUDA_OK(cudaMallocHost((void**)&b->sc_host, nsub * sizeof(PcgScalars)));
  BTRY(balloc(b, &b->iter_counter, 1));

  SFCDD_CUDA_OK(cudaEventRecord(e1, s));
  SFCDD_CUDA_OK(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  b->setup_ms = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (auto& a : b->allocs)
    if (a == keys || a == sort_tmp || a == tfirst) {
      cudaFree(a);
      a = nullptr;
    }
  ErrWord ew{};
  SFCDD_CUDA_OK(cudaMemcpy(&ew, b->err, sizeof(ErrWord), cudaMemcpyDeviceToHost));
  return ew.code;
}

void batch_destroy(sfcdd_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (void* p : b->allocs)
    if (p) cudaFree(p);
  if (b->sc_host) cudaFreeHost(b->sc_host);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
}

}  // namespace

extern "C" {

int sfcdd_batch_setup_each(const int* levels, const int* P, int nsub, int d, double overlap,
                           const sfcdd_options* opt, sfcdd_batch** out) {
  if (!out) return SFCDD_ERR_INVALID_ARG;
  *out = nullptr;
  sfcdd_batch* b = new (std::nothrow) sfcdd_batch();
  if (!b) return SFCDD_ERR_NOMEM;
  const int rc = batch_setup_impl(b, levels, nsub, d, P, overlap, opt);
  if (rc != SFCDD_OK) {
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    batch_destroy(b);
    return rc;
  }
  *out = b;
  return SFCDD_OK;
}

int sfcdd_batch_setup(const int* levels, int nsub, int d, int P, double overlap,
                      const sfcdd_options* opt, sfcdd_batch** out) {
  if (!out) return SFCDD_ERR_INVALID_ARG;
  *out = nullptr;
  if (nsub < 1) return SFCDD_ERR_INVALID_ARG;
  const std::vector<int> Ps(nsub, P);
  return sfcdd_batch_setup_each(levels, Ps.data(), nsub, d, overlap, opt, out);
}

int sfcdd_batch_combine(sfcdd_batch* b, const double* coef_host, const double* u_dev,
                        const double* points_dev, long long npts, double* out_dev) {
  if (!b || !coef_host || !u_dev || npts < 0 || (npts > 0 && (!points_dev || !out_dev)))
    return SFCDD_ERR_INVALID_ARG;
  if (npts == 0) return SFCDD_OK;
  for (int si = 0; si < b->nsub; ++si) {
    if (!(coef_host[si] == coef_host[si])) return SFCDD_ERR_INVALID_ARG;
    b->h_comb[si].coef = coef_host[si];
  }
  cudaStream_t s = b->stream;
  SFCDD_CUDA_OK(cudaMemcpyAsync(b->d_comb, b->h_comb.data(), b->nsub * sizeof(CombSub),
                                cudaMemcpyHostToDevice, s));
  const long long warps_per_block = 256 / 32;
  const long long blocks = std::min<long long>((npts + warps_per_block - 1) / warps_per_block,
                                               152LL * 64);
  SFCDD_DISPATCH_D(k_combine, b->d, (unsigned)blocks, 256, 0, s, b->d_comb, b->nsub, u_dev,
                   points_dev, npts, out_dev);
  SFCDD_CUDA_OK(cudaGetLastError());
  SFCDD_CUDA_OK(cudaStreamSynchronize(s));
  return SFCDD_OK;
}

int sfcdd_batch_offsets(const sfcdd_batch* b, long long* offsets_host) {
  if (!b || !offsets_host) return SFCDD_ERR_INVALID_ARG;
  for (int si = 0; si <= b->nsub; ++si) offsets_host[si] = b->offs[si];
  return SFCDD_OK;
}

int sfcdd_batch_solve(sfcdd_batch* b, const double* f_dev, double* u_dev, double rtol, int maxit,
                      sfcdd_stats* per_sub, sfcdd_stats* total) {
  NvtxRange nvtx("sfcdd batch solve");
  if (!b || !f_dev || !u_dev || !(rtol >= 0) || maxit < 1) return SFCDD_ERR_INVALID_ARG;
  cudaStream_t s = b->stream;
  BTRY(build_graph(b, maxit));
  cudaEvent_t e0, e1;
  SFCDD_CUDA_OK(cudaEventCreate(&e0));
  SFCDD_CUDA_OK(cudaEventCreate(&e1));
  SFCDD_CUDA_OK(cudaEventRecord(e0, s));
  const dim3 gsub((b->maxN + 255) / 256, b->nsub);
  k_b_lex_to_curve<<<gsub, 256, 0, s>>>(b->dsub, b->code, f_dev, b->b);
  k_b_init<<<b->nsub, BT, 0, s>>>(b->dsub, b->b, b->x, b->r, b->p, b->z, b->sc, rtol, b->flexible);
  k_b_restrict<<<b->nsub, BT, 0, s>>>(b->dsub, b->r, b->g0, b->sc);
  enqueue_apply(b, s);  // z_0 = C^{-1} r_0, beta = 0, p = z_0
  SFCDD_CUDA_OK(cudaMemsetAsync(b->iter_counter, 0, sizeof(int), s));
  SFCDD_CUDA_OK(cudaGraphLaunch(b->graph, s));  // every PCG iteration of every subgrid
  SFCDD_CUDA_OK(cudaEventRecord(e1, s));
  SFCDD_DISPATCH_D(k_b_true_res, b->d, b->nsub, BT, 0, s, b->dsub, b->code, b->invpad, b->b, b->x,
                   b->sc);
  k_b_curve_to_lex<<<gsub, 256, 0, s>>>(b->dsub, b->code, b->x, u_dev);
  SFCDD_CUDA_OK(cudaMemcpyAsync(b->sc_host, b->sc, b->nsub * sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
  SFCDD_CUDA_OK(cudaStreamSynchronize(s));
  SFCDD_CUDA_OK(cudaGetLastError());
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->solve_ms = ms;
  ErrWord ew{};
  SFCDD_CUDA_OK(cudaMemcpy(&ew, b->err, sizeof(ErrWord), cudaMemcpyDeviceToHost));
  int rc = ew.code;
  int maxits = 0, not_done = 0;
  double worst = 0.0, worst_true = 0.0;
  for (int si = 0; si < b->nsub; ++si) {
    const PcgScalars& c = b->sc_host[si];
    const int st = c.status ? c.status : (c.done ? SFCDD_OK : SFCDD_ERR_MAXIT);
    if (!c.done) ++not_done;
    if (rc == SFCDD_OK && st != SFCDD_OK) rc = st;
    maxits = std::max(maxits, c.iter);
    worst = std::max(worst, c.rel);
    worst_true = std::max(worst_true, c.true_rel);
    if (per_sub) {
      per_sub[si].iters = c.iter;
      per_sub[si].status = st;
      per_sub[si].fail_index = ew.index;
      per_sub[si].rel_res = c.rel;
      per_sub[si].true_rel_res = c.true_rel;
      per_sub[si].setup_ms = b->setup_ms;
      per_sub[si].solve_ms = ms;
    }
  }
  if (total) {
    total->iters = maxits;
    total->status = rc;
    total->fail_index = not_done;
    total->rel_res = worst;
    total->true_rel_res = worst_true;
    total->setup_ms = b->setup_ms;
    total->solve_ms = ms;
  }
  return rc;
}

int sfcdd_batch_autotune(sfcdd_batch* b, int reps, sfcdd_tuning* out) {
  if (!b || reps < 1) return SFCDD_ERR_INVALID_ARG;
  cudaStream_t s = b->stream;
  // a substitution pair over every subgrid: the batched triangular solves of
  // one PCG iteration, without the converged-subgrid early exit
  auto pair = [&]() {
    TrsvArgs af = batch_trsv_args(b, true), ab = batch_trsv_args(b, false);
    af.sc = nullptr;
    ab.sc = nullptr;
    launch_trsv_fwd(af, b->st, s);
    launch_trsv_bwd(ab, b->st, s);
  };
  SFCDD_CUDA_OK(cudaMemsetAsync(b->r, 0, (size_t)b->Ntot * sizeof(double), s));
  cudaEvent_t e0, e1;
  SFCDD_CUDA_OK(cudaEventCreate(&e0));
  SFCDD_CUDA_OK(cudaEventCreate(&e1));
  const int opts[4] = {1, 2, 4, 0};  // 0: whole-matrix local items
  int best_l = b->nsub_local, best_c = b->nsub_coarse, cand = 0, rc = SFCDD_OK;
  float best = -1.f;
  for (int il = 0; il < 4 && rc == SFCDD_OK; ++il)
    for (int ic = 0; ic < 3 && rc == SFCDD_OK; ++ic) {
      const int sl = opts[il], sc = opts[ic];
      if (b->st != Store::F64 && sc == 1) continue;  // 64-row FP64 stage: FP64 launches only
      if (sl == 0 && !whole_fits(b->st, b->max_nt_local)) continue;
      rc = batch_configure(b, sl, sc);
      if (rc != SFCDD_OK) break;
      for (int k = 0; k < 2; ++k) pair();
      cudaEventRecord(e0, s);
      for (int k = 0; k < reps; ++k) pair();
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = SFCDD_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ++cand;
      if (best < 0.f || ms < best) {
        best = ms;
        best_l = sl;
        best_c = sc;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SFCDD_OK) return rc;
  ErrWord e{};
  SFCDD_CUDA_OK(cudaMemcpyAsync(&e, b->err, sizeof(ErrWord), cudaMemcpyDeviceToHost, s));
  SFCDD_CUDA_OK(cudaStreamSynchronize(s));
  if (e.code != 0) return e.code;
  BTRY(batch_configure(b, best_l, best_c));
  if (out) {
    out->slabs_local = best_l == 0 ? -1 : best_l;
    out->slabs_coarse = best_c;
    out->apply_ms = best / reps;
    out->candidates = cand;
  }
  return SFCDD_OK;
}

int sfcdd_batch_info(const sfcdd_batch* b, long long* n_total, long long* factor_bytes,
                     double* setup_ms) {
  if (!b) return SFCDD_ERR_INVALID_ARG;
  if (n_total) *n_total = b->Ntot;
  if (factor_bytes) *factor_bytes = b->factor_bytes;
  if (setup_ms) *setup_ms = b->setup_ms;
  return SFCDD_OK;
}

int sfcdd_batch_destroy(sfcdd_batch* b) {
  if (!b) return SFCDD_ERR_INVALID_ARG;
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  batch_destroy(b);
  return SFCDD_OK;
}

}  // extern "C"
