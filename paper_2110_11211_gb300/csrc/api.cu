// C-ABI entry points: setup (Algorithm 1), PCG solve around the two-level
// additive Schwarz preconditioner (Algorithm 2, eq. addSW; Sec. 3.3), adjoint,
// and introspection for parity checks.
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <chrono>
#include <new>
#include <vector>

#include "sfcdd_internal.cuh"

using namespace sfcdd;

namespace sfcdd {
static thread_local int g_last_cuda_error = 0;
int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  g_last_cuda_error = (int)e;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return SFCDD_ERR_NOMEM;
  }
  fprintf(stderr, "sfcdd: CUDA error %s (%s) at %s:%d: %s\n", cudaGetErrorName(e),
          cudaGetErrorString(e), file, line, what);
  return SFCDD_ERR_CUDA;
}

int make_grid(const int* levels, int d, const double* coeffs, GridDev& g, long long& N, int& B) {
  if (!levels || d < 1 || d > MAXD) return SFCDD_ERR_INVALID_ARG;
  N = 1;
  B = 0;
  int nbits = 0;
  for (int j = 0; j < d; ++j) {
    if (levels[j] < 1 || levels[j] > 30) return SFCDD_ERR_INVALID_ARG;
    N *= (1ll << levels[j]) - 1;
    nbits = std::max(nbits, levels[j]);
    B += levels[j];
    if (coeffs && (!(coeffs[j] > 0) || !std::isfinite(coeffs[j]))) return SFCDD_ERR_INVALID_ARG;
  }
  if (d * nbits > 64) return SFCDD_ERR_KEY_OVERFLOW;
  if (B > 31 || N >= (1ll << 31)) return SFCDD_ERR_UNSUPPORTED;
  g = GridDev{};
  g.d = d;
  g.N = (int)N;
  g.nbits = nbits;
  int off = 0, stride = 1;
  for (int j = d - 1; j >= 0; --j) {
    g.lev[j] = levels[j];
    g.off[j] = off;
    off += levels[j];
    g.size[j] = (1 << levels[j]) - 1;
    g.stride[j] = stride;
    stride *= g.size[j];
  }
  g.diag = 0.0;
  for (int j = 0; j < d; ++j) {
    g.w[j] = (coeffs ? coeffs[j] : 1.0) * std::ldexp(1.0, 2 * levels[j]);
    g.diag += 2.0 * g.w[j];
  }
  return SFCDD_OK;
}

int paper_q(long long N, int P) {
  const long long fN = N / P;
  int e = 0;
  while ((2ll << e) <= fN) ++e;  // floor(log2 floor(N/P))
  const long long qq = 1ll << std::max(e - 4, 0);
  return (int)std::min<long long>(std::max<long long>(qq, 1), fN);
}

// eqs. sloc, enlarge, omegai.  gamma is read as the rational round(gamma 2^16) /
// 2^16 so ceil/floor(eta tilde N) are exact.
int partition_ranges(long long N, int P, double gamma, int weighting, std::vector<int>& start,
                     std::vector<int>& len, std::vector<double>& omega, int& gfloor) {
  const long long den = 1 << 16;
  const long long gnum = llround(gamma * (double)den);
  const int gf = (int)(gnum / den);
  const long long eta = gnum % den;
  gfloor = gf;
  if (gnum <= 0 || 2 * gf + 1 >= P || P > N) return SFCDD_ERR_INVALID_ARG;
  const long long f = N / P, rr = N % P;
  auto tsize = [&](int t) { return t < rr ? f + 1 : f; };
  auto toff = [&](int t) { return t < rr ? t * (f + 1) : rr * (f + 1) + (t - rr) * f; };
  start.assign(P, 0);
  len.assign(P, 0);
  for (int i = 0; i < P; ++i) {
    const int left = ((i - gf - 1) % P + P) % P;
    const int right = (i + gf + 1) % P;
    const long long nl = (eta * tsize(left) + den - 1) / den;
    const long long nr = (eta * tsize(right)) / den;
    long long core = 0;
    for (int k = -gf; k <= gf; ++k) core += tsize(((i + k) % P + P) % P);
    const long long l = nl + core + nr;
    if (l > N) return SFCDD_ERR_INVALID_ARG;
    start[i] = (int)((toff(left) + tsize(left) - nl) % N);
    len[i] = (int)l;
  }
  // coverage counts are constant between range end points: sweep the segments
  std::vector<long long> cuts;
  cuts.reserve(2 * P + 2);
  cuts.push_back(0);
  cuts.push_back(N);
  for (int i = 0; i < P; ++i) {
    cuts.push_back(start[i]);
    cuts.push_back((start[i] + len[i]) % N);
  }
  std::sort(cuts.begin(), cuts.end());
  cuts.erase(std::unique(cuts.begin(), cuts.end()), cuts.end());
  const int nseg = (int)cuts.size() - 1;
  std::vector<int> cnt(nseg, 0);
  std::vector<std::pair<int, int>> segs(P);  // (first segment, number of segments)
  for (int i = 0; i < P; ++i) {
    const int a = (int)(std::lower_bound(cuts.begin(), cuts.end(), (long long)start[i]) -
                        cuts.begin());
    long long covered = 0;
    int k = a, nsg = 0;
    while (covered < len[i]) {
      cnt[k] += 1;
      covered += cuts[k + 1] - cuts[k];
      k = (k + 1) % nseg;
      ++nsg;
    }
    segs[i] = {a, nsg};
  }
  omega.assign(P, 1.0);
  if (weighting == SFCDD_WEIGHT_OMEGA) {
    for (int i = 0; i < P; ++i) {
      int mn = 1 << 30;
      for (int k = 0; k < segs[i].second; ++k) mn = std::min(mn, cnt[(segs[i].first + k) % nseg]);
      omega[i] = 1.0 / (double)mn;
    }
  }
  return SFCDD_OK;
}

void build_worklists(const std::vector<int>& nt, const std::vector<char>& include,
                     const std::vector<int>& nsub, std::vector<TrsvWork>& wf,
                     std::vector<TrsvWork>& wb) {
  struct Item {
    long long num, den;  // progress (r + 1) / nt as an exact fraction
    int m, r, s;
  };
  std::vector<Item> items;
  for (int m = 0; m < (int)nt.size(); ++m)
    if (include[m]) {
      if (nsub[m] == 0) {
        items.push_back({0, 1, m, -1, 0});  // whole matrix: depends on nothing, taken first
        continue;
      }
      for (int r = 0; r < nt[m]; ++r)
        for (int sl = 0; sl < nsub[m]; ++sl) items.push_back({r + 1, nt[m], m, r, sl});
    }
  std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& b) {
    const long long l = a.num * b.den, rr = b.num * a.den;
    return l != rr ? l < rr : a.m < b.m;
  });
  wf.clear();
  wb.clear();
  for (const Item& it : items) {
    wf.push_back({it.m, it.r, it.s});
    wb.push_back({it.m, it.r < 0 ? -1 : nt[it.m] - 1 - it.r, it.s});
  }
}

// Reverse Cuthill-McKee numbering of an undirected graph given as adjacency
// lists adj[v * stride + k], k < deg[v]: per connected component a breadth-first
// sweep from a pseudo-peripheral node (repeated sweeps from a minimum-degree
// node of the last level while the number of levels grows), neighbours taken
// by increasing degree (ties by index); the concatenated order is reversed.
// order[r] = node numbered r.  Deterministic.
void rcm_order(int n, const std::vector<int>& deg, const std::vector<int>& adj, int stride,
               std::vector<int>& order) {
  // neighbour lists in one flat array, each sorted by (degree, index)
  std::vector<int> off(n + 1, 0);
  for (int v = 0; v < n; ++v) off[v + 1] = off[v] + deg[v];
  std::vector<int> nb(off[n]);
  for (int v = 0; v < n; ++v) {
    int* l = nb.data() + off[v];
    std::copy(adj.begin() + (size_t)v * stride, adj.begin() + (size_t)v * stride + deg[v], l);
    std::sort(l, l + deg[v], [&](int a, int b) { return deg[a] != deg[b] ? deg[a] < deg[b] : a < b; });
  }
  std::vector<int> stamp(n, -1), queue(n);
  int stampv = 0;
  // number of breadth-first levels from root; last = min-degree node of the last level
  auto sweep = [&](int root, int& last) {
    ++stampv;
    int head = 0, tail = 0, lev_begin = 0, nlev = 0;
    queue[tail++] = root;
    stamp[root] = stampv;
    while (head < tail) {
      lev_begin = head;
      const int lev_end = tail;
      ++nlev;
      for (; head < lev_end; ++head) {
        const int v = queue[head];
        for (int k = off[v]; k < off[v + 1]; ++k) {
          const int u = nb[k];
          if (stamp[u] != stampv) {
            stamp[u] = stampv;
            queue[tail++] = u;
          }
        }
      }
    }
    last = queue[lev_begin];
    for (int k = lev_begin; k < tail; ++k) {
      const int v = queue[k];
      if (deg[v] < deg[last] || (deg[v] == deg[last] && v < last)) last = v;
    }
    return nlev;
  };
  std::vector<char> seen(n, 0);
  order.clear();
  order.reserve(n);
  for (int s0 = 0; s0 < n; ++s0) {
    if (seen[s0]) continue;
    int root = s0, levels = 0;
    for (int it = 0; it < 8; ++it) {
      int last;
      const int l = sweep(root, last);
      if (l <= levels) break;
      levels = l;
      root = last;
    }
    size_t head = order.size();
    order.push_back(root);
    seen[root] = 1;
    while (head < order.size()) {
      const int v = order[head++];
      for (int k = off[v]; k < off[v + 1]; ++k) {
        const int u = nb[k];
        if (!seen[u]) {
          seen[u] = 1;
          order.push_back(u);
        }
      }
    }
  }
  std::reverse(order.begin(), order.end());
}

void build_skyline(const std::vector<int>& nt, const std::vector<int>& vbase,
                   const std::vector<char>& is_coarse, const std::vector<int>& cb,
                   const std::vector<int>& tfirst, SkylineHost& o) {
  const int nmat = (int)nt.size();
  const int nrows = (int)tfirst.size();
  o.kmin.assign(nrows, 0);
  o.rowoff.assign(nrows, 0);
  for (int r = 0; r < nrows; ++r) o.kmin[r] = tfirst[r] / TILE;
  // a matrix solved with cb-tile diagonal blocks keeps whole blocks in every row
  for (int m = 0; m < nmat; ++m) {
    const int fb = vbase[m] / TILE;
    if (cb[m] > 1)
      for (int I = 0; I < nt[m]; ++I) o.kmin[fb + I] = o.kmin[fb + I] / cb[m] * cb[m];
  }
  std::vector<int> colcnt(nrows, 0);
  o.stored.assign(nmat, 0);
  o.tbase.assign(nmat, 0);
  int max_nt_l = 1, max_nt_c = 1;
  for (int m = 0; m < nmat; ++m) {
    const int fb = vbase[m] / TILE;
    int off = 0;
    for (int I = 0; I < nt[m]; ++I) {
      o.rowoff[fb + I] = off;
      off += I - o.kmin[fb + I] + 1;
      for (int K = o.kmin[fb + I]; K < I; ++K) colcnt[fb + K] += 1;
    }
    o.stored[m] = off;
    if (is_coarse[m]) {
      o.tbase[m] = o.ctiles * TILE2;
      o.ctiles += off;
      o.max_ctiles = std::max(o.max_ctiles, off);
      max_nt_c = std::max(max_nt_c, nt[m]);
    } else {
      o.tbase[m] = o.ltiles * TILE2;
      o.ltiles += off;
      o.max_ltiles = std::max(o.max_ltiles, off);
      max_nt_l = std::max(max_nt_l, nt[m]);
    }
  }
  o.colptr.assign(nrows + 1, 0);
  for (int r = 0; r < nrows; ++r) o.colptr[r + 1] = o.colptr[r] + colcnt[r];
  o.colidx.assign(std::max(o.colptr[nrows], 1), 0);
  std::vector<int> pos(o.colptr.begin(), o.colptr.end() - 1);
  for (int m = 0; m < nmat; ++m) {
    const int fb = vbase[m] / TILE;
    for (int I = 0; I < nt[m]; ++I)
      for (int K = o.kmin[fb + I]; K < I; ++K) o.colidx[pos[fb + K]++] = I;
  }
  // tiles the substitutions stream: forward rows skip their own diagonal block,
  // backward rows read their block of E tiles and the column tiles below it
  for (int m = 0; m < nmat; ++m) {
    const int fb = vbase[m] / TILE;
    long long f = 0, b = 0;
    for (int I = 0; I < nt[m]; ++I) {
      const int blk0 = I / cb[m] * cb[m];
      const int blk1 = std::min(blk0 + cb[m], nt[m]);
      f += std::max(0, blk0 - o.kmin[fb + I]);
      b += blk1 - blk0;
      for (int k = o.colptr[fb + I]; k < o.colptr[fb + I + 1]; ++k)
        if (o.colidx[k] >= blk1) ++b;
    }
    (is_coarse[m] ? o.fwd_tiles_c : o.fwd_tiles_l) += f;
    (is_coarse[m] ? o.bwd_tiles_c : o.bwd_tiles_l) += b;
  }
  o.col_max_local.assign(max_nt_l, 0);
  o.col_max_coarse.assign(max_nt_c, 0);
  const double t3 = (double)TILE * TILE * TILE;
  for (int m = 0; m < nmat; ++m) {
    const int fb = vbase[m] / TILE;
    for (int K = 0; K < nt[m]; ++K) {
      const int c = colcnt[fb + K];
      const double po = 2.0 * t3 / 3.0, tr = c * 2.0 * t3, sy = c * (c + 1) / 2.0 * 2.0 * t3;
      if (is_coarse[m]) {
        o.col_max_coarse[K] = std::max(o.col_max_coarse[K], c);
        o.coarse += po + tr + sy;
      } else {
        o.col_max_local[K] = std::max(o.col_max_local[K], c);
        o.potrf += po;
        o.trsm += tr;
        o.syrk += sy;
      }
    }
  }
}

}  // namespace sfcdd

struct sfcdd_handle {
  // problem
  int d = 0;
  int lev[MAXD] = {0};
  double coeffs[MAXD] = {0};
  int N = 0, nbits = 0, B = 0, P = 0, q = 0, N0 = 0, gfloor = 0;
  double gamma = 0;
  int precision = 0, variant = 0, weighting = 1, flexible = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t side_stream = nullptr;  // coarse factorization, concurrent with the local one
  GridDev g{};
  PartDev pd{};
  std::vector<int> h_start, h_len;
  std::vector<double> h_omega;
  // curve
  unsigned* curve_code = nullptr;
  int* invpad = nullptr;
  int *d_start = nullptr, *d_len = nullptr;
  double* d_omega = nullptr;
  // tiles (P locals + 1 coarse)
  std::vector<int> h_n, h_nt, h_vbase;
  std::vector<long long> h_tbase;
  int *d_n = nullptr, *d_nt = nullptr, *d_vbase = nullptr;
  long long* d_tbase = nullptr;
  long long* d_zero64 = nullptr;
  int *d_kmin = nullptr, *d_rowoff = nullptr, *d_colptr = nullptr, *d_colidx = nullptr;
  MatDesc* d_md = nullptr;
  int* d_lperm = nullptr;
  int* d_linv = nullptr;
  int* d_crow = nullptr;    // coarse block -> coarse factor row
  int* d_cblock = nullptr;  // coarse factor row -> coarse block
  int local_order = 0;
  std::vector<int> h_kmin, h_rowoff, stored, col_max_local, col_max_coarse;
  TileSetDev ts{};
  Store st = Store::F64;
  void* ltiles = nullptr;   // Lh tiles of the local factors
  void* lut = nullptr;      // Lh^T tiles, E_K on the diagonal
  double* ctiles = nullptr;
  double* cut = nullptr;
  long long ltile_elems = 0, ctile_elems = 0;
  int max_nt = 0, nt0 = 0, max_ltiles = 0, max_ctiles = 0;
  int nsub_local = 1, nsub_coarse = 4;
  bool tensor_cores = false;  // factorization tile products on tcgen05 (FP32 split / FP64 sliced)
  bool bf16_operands = false; // BF16 local factors: bf16 operands (kind::f16), else the TF32 split
  int cb_coarse = 4;  // tiles per unit diagonal block of the coarse substitution form
  long long fwd_tiles_l = 0, bwd_tiles_l = 0, fwd_tiles_c = 0, bwd_tiles_c = 0;
  // local factor elements the substitutions need (nonzero rows of the off-block
  // tiles, whole E tiles), from the zero-row bounds nzr
  int* d_nzr = nullptr;
  std::vector<int> h_nzr;
  long long fwd_elems_l = 0, bwd_elems_l = 0;
  // substitution work lists (each with its own ticket counters: the items of a
  // launch map to tickets modulo the list length): the variant's matrices, and
  // for the balanced variant the local matrices and the coarse matrix alone
  struct WorkList {
    TrsvWork *f = nullptr, *b = nullptr;
    int n = 0;
    unsigned long long *tf = nullptr, *tb = nullptr;
  } lists[3];
  double *ybuf = nullptr, *dbuf = nullptr, *zcbuf = nullptr;
  double* bal[4] = {nullptr, nullptr, nullptr, nullptr};  // balanced apply: w, g - A w, t, v
  long long vtotal = 0;
  // PCG
  double *b = nullptr, *x = nullptr, *r = nullptr, *p = nullptr, *qv = nullptr, *z = nullptr,
         *tmp = nullptr, *tmp2 = nullptr, *g0 = nullptr;
  PcgScalars* sc = nullptr;
  PcgScalars* sc_host = nullptr;
  ReduceWs ws{};
  // the vector phase of an iteration as one cooperative launch (every variant
  // but the balanced one): CTA ranges, barrier, partials, the second p buffer
  bool fused = false;
  int fused_rc = 0;
  FusedPcg fz{};
  double* p2 = nullptr;
  ErrWord* err = nullptr;
  cudaGraphExec_t iter_graph = nullptr;
  int graph_kernels[SFCDD_K_COUNT] = {0};
  // accounting
  bool profiling = false;
  bool auto_local = false;  // slabs_local left to the library: whole-matrix items when they fit
  long long launches[SFCDD_K_COUNT] = {0};
  double ms[SFCDD_K_COUNT] = {0};
  double setup_ms = 0, solve_ms = 0;
  double factor_flops = 0;
  double work_potrf = 0, work_trsm = 0, work_syrk = 0, work_coarse = 0;
  std::vector<void*> allocs;
};

namespace {

template <class T>
int dalloc(sfcdd_handle* h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? SFCDD_ERR_NOMEM : SFCDD_ERR_CUDA;
  }
  h->allocs.push_back((void*)*p);
  return SFCDD_OK;
}

// Slab counts the substitution kernel is built for: local rows of 64, 32 or 16,
// coarse rows of 64, 32 or 16.  FP32 / BF16 launches size their shared memory
// for the local tiles, so a full 64-row FP64 coarse stage needs an FP64 launch.
bool valid_slabs(int precision, int nsub_local, int nsub_coarse) {
  // nsub_local 0: one CTA per local matrix (whole-matrix sweeps)
  const bool l = nsub_local == 0 || nsub_local == 1 || nsub_local == 2 || nsub_local == 4;
  const bool c = nsub_coarse == 1 || nsub_coarse == 2 || nsub_coarse == 4;
  return l && c && (precision == SFCDD_FP64 || nsub_coarse != 1);
}

void dfree(sfcdd_handle* h, void* p) {
  if (!p) return;
  for (auto& a : h->allocs)
    if (a == p) {
      cudaFree(p);
      a = nullptr;
    }
}

#define TRY(x)                  \
  do {                          \
    int _rc = (x);              \
    if (_rc != SFCDD_OK) return _rc; \
  } while (0)

// Launch accounting: counts launches per class and, when profiling, brackets
// each launch with CUDA events on the launching stream.
struct Prof : LaunchHook {
  sfcdd_handle* h;
  cudaStream_t s;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> evs;
  cudaEvent_t pending = nullptr;
  Prof(sfcdd_handle* h_, cudaStream_t s_) : h(h_), s(s_) {}
  void before(int cls) override {
    h->launches[cls] += 1;
    if (h->profiling) {
      cudaEventCreate(&pending);
      cudaEventRecord(pending, s);
    }
  }
  void after(int cls) override {
    if (h->profiling && pending) {
      cudaEvent_t b;
      cudaEventCreate(&b);
      cudaEventRecord(b, s);
      evs.push_back({cls, {pending, b}});
      pending = nullptr;
    }
  }
  template <class F>
  void run(int cls, F&& f) {
    before(cls);
    f();
    after(cls);
  }
  void collect() {
    for (auto& e : evs) {
      cudaEventSynchronize(e.second.second);
      float t = 0.f;
      cudaEventElapsedTime(&t, e.second.first, e.second.second);
      h->ms[e.first] += t;
      cudaEventDestroy(e.second.first);
      cudaEventDestroy(e.second.second);
    }
    evs.clear();
  }
  ~Prof() override { collect(); }
};

// Routes every factorization class of the coarse matrix to one class.
struct CoarseHook : LaunchHook {
  Prof& p;
  explicit CoarseHook(Prof& p_) : p(p_) {}
  void before(int) override { p.before(SFCDD_K_COARSE_FACTOR); }
  void after(int) override { p.after(SFCDD_K_COARSE_FACTOR); }
};

enum { LIST_MAIN = 0, LIST_LOCAL = 1, LIST_COARSE = 2 };

// Local factor elements each substitution needs, from the zero-row bounds:
// forward, the nonzero rows of the off-block Lh tiles; backward, the E tile of
// every row and the nonzero columns of the Lh^T tiles (the same elements).
static int count_local_elems(sfcdd_handle* h) {
  const int P = h->P;
  if (h->variant == SFCDD_COARSE_ONLY) return SFCDD_OK;
  const int nrows = (int)h->h_nzr.size();
  SFCDD_CUDA_OK(cudaMemcpy(h->h_nzr.data(), h->d_nzr, nrows * sizeof(int), cudaMemcpyDeviceToHost));
  long long off = 0, diag = 0;
  for (int m = 0; m < P; ++m) {
    const int fb = h->h_vbase[m] / TILE;
    for (int I = 0; I < h->h_nt[m]; ++I) {
      off += (long long)(I - h->h_kmin[fb + I]) * h->h_nzr[fb + I] * TILE;
      diag += TILE2;
    }
  }
  h->fwd_elems_l = off;
  h->bwd_elems_l = off + diag;
  return SFCDD_OK;
}

TrsvArgs trsv_args(sfcdd_handle* h, bool fwd, const double* rhs, const PcgScalars* sc,
                   int list = LIST_MAIN) {
  TrsvArgs a{};
  a.ts = h->ts;
  a.md = h->d_md;
  a.ltiles = h->ltiles;
  a.lut = h->lut;
  a.ctiles = h->ctiles;
  a.cut = h->cut;
  a.rhs = rhs;
  a.g0 = h->g0;
  a.cblock = h->pd.cblock;
  a.y = h->ybuf;
  a.dout = h->dbuf;
  a.zc = h->zcbuf;
  const auto& wl = h->lists[list];
  a.work = fwd ? wl.f : wl.b;
  a.nwork = wl.n;
  a.ticket = fwd ? wl.tf : wl.tb;
  a.err = h->err;
  a.sc = sc;
  if (h->nsub_local == 0 && list != LIST_COARSE) a.zv_doubles = h->max_nt * TILE;
  a.wide_ring = 1;
  return a;
}

// One-matrix views (tile base 0) of the coarse matrix and of local matrix i.
TileSetDev coarse_view(const sfcdd_handle* h) {
  TileSetDev v = h->ts;
  v.lperm = nullptr;  // the local numbering does not apply to the coarse matrix
  v.linv = nullptr;
  v.nmat = 1;
  v.n = h->d_n + h->P;
  v.nt = h->d_nt + h->P;
  v.vbase = h->d_vbase + h->P;
  v.tbase = h->d_zero64;
  return v;
}
TileSetDev local_view(const sfcdd_handle* h, int i) {
  TileSetDev v = h->ts;
  v.nmat = 1;
  v.n = h->d_n + i;
  v.nt = h->d_nt + i;
  v.vbase = h->d_vbase + i;
  v.tbase = h->d_zero64;
  return v;
}

int prolong_mode(const sfcdd_handle* h) {
  if (h->variant == SFCDD_ONE_LEVEL) return 1;
  if (h->variant == SFCDD_COARSE_ONLY) return 2;
  return 0;
}

// One substitution pair (forward, backward) over a work list; local right-hand
// sides sliced from g, the coarse one from g0.
void enqueue_solves(sfcdd_handle* h, Prof& pf, const double* g, PcgScalars* sc, int list) {
  cudaStream_t s = pf.s;
  TrsvArgs af = trsv_args(h, true, g, sc, list);
  TrsvArgs ab = trsv_args(h, false, g, sc, list);
  pf.run(SFCDD_K_TRSV_FWD, [&] { launch_trsv_fwd(af, h->st, s); });
  pf.run(SFCDD_K_TRSV_BWD, [&] { launch_trsv_bwd(ab, h->st, s); });
}

// w = F g = R_0^T A_0^{-1} R_0 g
void enqueue_coarse_correction(sfcdd_handle* h, Prof& pf, const double* g, double* w,
                               PcgScalars* sc) {
  cudaStream_t s = pf.s;
  pf.run(SFCDD_K_RESTRICT, [&] { launch_restrict(h->pd, g, h->g0, sc, s); });
  enqueue_solves(h, pf, g, sc, LIST_COARSE);
  pf.run(SFCDD_K_PROLONG,
         [&] { launch_prolong(h->pd, h->ts, 2, h->dbuf, g, w, sc, h->ws, s, false); });
}

// Balanced variant (eq. balSW): z = G^T C_(1) G g + F g with G = I - A F and
// G^T = I - F A (A, F symmetric), C_(1) the weighted one-level operator:
//   w = F g,  t = C_(1) (g - A w),  v = F A t,  z = t - v + w.
void enqueue_apply_balanced(sfcdd_handle* h, Prof& pf, const double* g, double* z,
                            PcgScalars* sc) {
  cudaStream_t s = pf.s;
  double *w = h->bal[0], *gg = h->bal[1], *t = h->bal[2], *v = h->bal[3];
  enqueue_coarse_correction(h, pf, g, w, sc);
  pf.run(SFCDD_K_STENCIL,
         [&] { launch_residual(h->g, h->curve_code, h->invpad, g, w, gg, sc, h->ws, s); });
  enqueue_solves(h, pf, gg, sc, LIST_LOCAL);
  pf.run(SFCDD_K_PROLONG,
         [&] { launch_prolong(h->pd, h->ts, 1, h->dbuf, gg, t, sc, h->ws, s, false); });
  pf.run(SFCDD_K_STENCIL,
         [&] { launch_stencil(h->g, h->curve_code, h->invpad, t, h->tmp2, 0, sc, h->ws, s); });
  enqueue_coarse_correction(h, pf, h->tmp2, v, sc);
  pf.run(SFCDD_K_VECTOR, [&] { launch_combine_bal(h->N, t, v, w, g, z, sc, h->ws, s); });
}

// z = C^{-1} g in curve order.  With sc != null the prolongation finalizes r^T z
// (PCG) and every kernel returns early once the solve has converged.
void enqueue_apply(sfcdd_handle* h, Prof& pf, const double* g, double* z, PcgScalars* sc) {
  cudaStream_t s = pf.s;
  if (h->variant == SFCDD_BALANCED) {
    enqueue_apply_balanced(h, pf, g, z, sc);
    return;
  }
  const bool coarse = h->variant != SFCDD_ONE_LEVEL;
  if (coarse) pf.run(SFCDD_K_RESTRICT, [&] { launch_restrict(h->pd, g, h->g0, sc, s); });
  enqueue_solves(h, pf, g, sc, LIST_MAIN);
  pf.run(SFCDD_K_PROLONG, [&] {
    launch_prolong(h->pd, h->ts, prolong_mode(h), h->dbuf, g, z, sc, h->ws, s);
  });
}

void enqueue_iteration(sfcdd_handle* h, Prof& pf) {
  cudaStream_t s = pf.s;
  if (h->fused) {
    // z = C^{-1} r through the substitutions (g0 = R_0 r was formed by the
    // previous vector phase), then the whole vector phase in one launch
    enqueue_solves(h, pf, h->r, h->sc, LIST_MAIN);
    pf.run(SFCDD_K_PCG_VECTOR, [&] { h->fused_rc = launch_fused_pcg(h->fz, s); });
    return;
  }
  pf.run(SFCDD_K_STENCIL,
         [&] { launch_stencil(h->g, h->curve_code, h->invpad, h->p, h->qv, 1, h->sc, h->ws, s); });
  pf.run(SFCDD_K_UPDATE, [&] { launch_update_xr(h->N, h->x, h->r, h->p, h->qv, h->sc, h->ws, s); });
  enqueue_apply(h, pf, h->r, h->z, h->sc);
  pf.run(SFCDD_K_VECTOR, [&] { launch_update_p(h->N, h->z, h->p, h->sc, s); });
}

// Substitution work items: the per-matrix descriptors (slab counts: local rows
// of 64 / nsub_local, coarse rows of 64 / nsub_coarse) and the work lists of
// tile-row slabs in dependency-safe order.  Re-running it with other slab
// counts replaces both and drops the captured iteration graph.
int configure_substitution(sfcdd_handle* h, int nsub_local, int nsub_coarse) {
  const int P = h->P;
  cudaStream_t s = h->stream;
  if (nsub_local == 0 && (!whole_fits(h->st, h->max_nt) || !h->d_nzr)) return SFCDD_ERR_INVALID_ARG;
  SFCDD_CUDA_OK(cudaStreamSynchronize(s));
  if (h->iter_graph) {
    cudaGraphExecDestroy(h->iter_graph);
    h->iter_graph = nullptr;
  }
  h->nsub_local = nsub_local;
  h->nsub_coarse = nsub_coarse;
  std::vector<MatDesc> md(P + 1);
  for (int m = 0; m < P; ++m) md[m] = {0, h->N, h->h_start[m], 0, 0, nsub_local, 1};
  md[P] = {0, h->N0, 0, 1, 0, nsub_coarse, h->cb_coarse};
  if (!h->d_md) TRY(dalloc(h, &h->d_md, P + 1));
  SFCDD_CUDA_OK(cudaMemcpyAsync(h->d_md, md.data(), (P + 1) * sizeof(MatDesc), cudaMemcpyHostToDevice, s));
  std::vector<int> nsub(P + 1, nsub_local);
  nsub[P] = nsub_coarse;
  for (int li = 0; li < 3; ++li) {
    std::vector<char> include(P + 1, 1);
    if (li == LIST_MAIN) {
      if (h->variant == SFCDD_COARSE_ONLY)
        for (int m = 0; m < P; ++m) include[m] = 0;
      if (h->variant == SFCDD_ONE_LEVEL) include[P] = 0;
    } else {
      if (h->variant != SFCDD_BALANCED) continue;
      if (li == LIST_LOCAL) include[P] = 0;
      else
        for (int m = 0; m < P; ++m) include[m] = 0;
    }
    std::vector<TrsvWork> wf, wb;
    build_worklists(h->h_nt, include, nsub, wf, wb);
    auto& wl = h->lists[li];
    dfree(h, wl.f);
    dfree(h, wl.b);
    wl.n = (int)wf.size();
    TRY(dalloc(h, &wl.f, wl.n));
    TRY(dalloc(h, &wl.b, wl.n));
    SFCDD_CUDA_OK(cudaMemcpyAsync(wl.f, wf.data(), wf.size() * sizeof(TrsvWork), cudaMemcpyHostToDevice, s));
    SFCDD_CUDA_OK(cudaMemcpyAsync(wl.b, wb.data(), wb.size() * sizeof(TrsvWork), cudaMemcpyHostToDevice, s));
    if (!wl.tf) TRY(dalloc(h, &wl.tf, 1));
    if (!wl.tb) TRY(dalloc(h, &wl.tb, 1));
    SFCDD_CUDA_OK(cudaMemsetAsync(wl.tf, 0, sizeof(unsigned long long), s));
    SFCDD_CUDA_OK(cudaMemsetAsync(wl.tb, 0, sizeof(unsigned long long), s));
    SFCDD_CUDA_OK(cudaStreamSynchronize(s));  // host vectors go out of scope
  }
  return SFCDD_OK;
}

int build_graph(sfcdd_handle* h) {
  if (h->iter_graph) return SFCDD_OK;
  long long before[SFCDD_K_COUNT];
  memcpy(before, h->launches, sizeof(before));
  const bool prof = h->profiling;
  h->profiling = false;
  SFCDD_CUDA_OK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  Prof pf(h, h->cap_stream);
  h->fused_rc = 0;
  enqueue_iteration(h, pf);
  cudaGraph_t graph;
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
  if (h->fused_rc) {
    if (e == cudaSuccess) cudaGraphDestroy(graph);
    h->profiling = prof;
    return h->fused_rc;
  }
  h->profiling = prof;
  for (int k = 0; k < SFCDD_K_COUNT; ++k) {
    h->graph_kernels[k] = (int)(h->launches[k] - before[k]);
    h->launches[k] = before[k];
  }
  SFCDD_CUDA_OK(e);
  e = cudaGraphInstantiate(&h->iter_graph, graph, 0);
  cudaGraphDestroy(graph);
  SFCDD_CUDA_OK(e);
  return SFCDD_OK;
}

int check_err(sfcdd_handle* h, int* fail_index) {
  ErrWord e{};
  SFCDD_CUDA_OK(cudaMemcpyAsync(&e, h->err, sizeof(ErrWord), cudaMemcpyDeviceToHost, h->stream));
  SFCDD_CUDA_OK(cudaStreamSynchronize(h->stream));
  if (fail_index) *fail_index = e.index;
  return e.code;
}

// The fused vector phase: CTA count (resident in one cooperative launch, at
// most one CTA per 256 points and, with a coarse space, per coarse block) and
// the CTA ranges of curve positions (whole coarse blocks when there is a
// coarse space, so the restriction stays inside a CTA).
int setup_fused(sfcdd_handle* h) {
  const int mode = prolong_mode(h);
  int nb = fused_pcg_blocks(h->d);
  if (nb <= 0) return SFCDD_ERR_CUDA;
  nb = std::min(nb, std::max(1, (h->N + 255) / 256));
  if (mode != 1) nb = std::min(nb, h->N0);
  std::vector<int> range(nb + 1);
  for (int c = 0; c <= nb; ++c) {
    if (mode == 1) {
      range[c] = (int)((long long)h->N * c / nb);
    } else {
      const int b = (int)((long long)h->N0 * c / nb);
      int st = h->N, sz = 0;
      if (b < h->N0) coarse_block_range(h->pd, b, st, sz);
      range[c] = st;
    }
  }
  FusedPcg& f = h->fz;
  f.nblocks = nb;
  f.mode = mode;
  int* d_range = nullptr;
  TRY(dalloc(h, &d_range, nb + 1));
  TRY(dalloc(h, &f.bar, 2));
  TRY(dalloc(h, &f.part, (size_t)4 * nb));
  TRY(dalloc(h, &f.ws.partial, (size_t)2 * nb));
  TRY(dalloc(h, &f.ws.counter, 1));
  TRY(dalloc(h, &h->p2, h->N));
  cudaStream_t s = h->stream;
  SFCDD_CUDA_OK(cudaMemcpyAsync(d_range, range.data(), (nb + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemsetAsync(f.bar, 0, 2 * sizeof(unsigned), s));
  SFCDD_CUDA_OK(cudaMemsetAsync(f.ws.counter, 0, sizeof(unsigned), s));
  SFCDD_CUDA_OK(cudaStreamSynchronize(s));  // the host range vector goes out of scope
  f.ws.nblocks = nb;
  f.range = d_range;
  f.g = h->g;
  f.pd = h->pd;
  f.ts = h->ts;
  f.code = h->curve_code;
  f.invpad = h->invpad;
  f.dvec = h->dbuf;
  f.x = h->x;
  f.r = h->r;
  f.z = h->z;
  f.p[0] = h->p;
  f.p[1] = h->p2;
  f.q = h->qv;
  f.g0 = h->g0;
  f.sc = h->sc;
  f.err = h->err;
  h->fused = true;
  return SFCDD_OK;
}

// ---------------------------------------------------------------------------
// Host-side partition of one problem into the handle.
int build_partition(sfcdd_handle* h) {
  return partition_ranges(h->N, h->P, h->gamma, h->weighting, h->h_start, h->h_len, h->h_omega,
                          h->gfloor);
}

int setup_impl(sfcdd_handle* h, const int* levels, int d, int P, double overlap,
               const sfcdd_options* opt) {
  NvtxRange nvtx("sfcdd setup");
  if (!levels || d < 1 || d > MAXD || P < 2 || !(overlap > 0)) return SFCDD_ERR_INVALID_ARG;
  h->d = d;
  long long N = 1;
  int B = 0;
  {
    const int rc = make_grid(levels, d, opt ? opt->coeffs : nullptr, h->g, N, B);
    if (rc != SFCDD_OK) return rc;
  }
  const int nbits = h->g.nbits;
  for (int j = 0; j < d; ++j) {
    h->lev[j] = levels[j];
    h->coeffs[j] = (opt && opt->coeffs) ? opt->coeffs[j] : 1.0;
  }
  if (P > N) return SFCDD_ERR_INVALID_ARG;
  h->N = (int)N;
  h->nbits = nbits;
  h->B = B;
  h->P = P;
  h->gamma = overlap;
  sfcdd_options o;
  sfcdd_default_options(&o);
  if (opt) o = *opt;
  h->precision = o.precision;
  h->variant = o.variant;
  h->weighting = o.weighting;
  if (h->precision < 0 || h->precision > 2 || h->variant < 0 || h->variant > 3 ||
      h->weighting < 0 || h->weighting > 1)
    return SFCDD_ERR_INVALID_ARG;
  // public -1: one CTA per local matrix (internal 0); 0: decided once the tile
  // rows are known
  h->auto_local = o.slabs_local == 0;
  h->nsub_local = o.slabs_local == 0 ? 1 : (o.slabs_local == -1 ? 0 : o.slabs_local);
  h->nsub_coarse = o.slabs_coarse == 0 ? 2 : o.slabs_coarse;
  h->cb_coarse = o.coarse_block == 0 ? 4 : o.coarse_block;
  if (h->cb_coarse != 1 && h->cb_coarse != 2 && h->cb_coarse != 4 && h->cb_coarse != 8)
    return SFCDD_ERR_INVALID_ARG;
  if (!valid_slabs(h->precision, h->nsub_local, h->nsub_coarse)) return SFCDD_ERR_INVALID_ARG;
  if (o.tensor_cores < -1 || o.tensor_cores > 2) return SFCDD_ERR_INVALID_ARG;
  h->tensor_cores = o.tensor_cores != 0;
  h->bf16_operands = h->precision == SFCDD_BF16 && h->tensor_cores && o.tensor_cores != 2;
  h->flexible = o.flexible < 0 ? (h->precision != SFCDD_FP64 ? 1 : 0) : (o.flexible ? 1 : 0);
  h->stream = (cudaStream_t)o.stream;
  h->profiling = o.profile != 0;
  const long long fN = N / P;
  h->q = o.q <= 0 ? paper_q(N, P) : o.q;
  if (h->q < 1 || h->q > fN) return SFCDD_ERR_INVALID_ARG;
  h->N0 = h->q * P;
  h->st = (Store)h->precision;

  SFCDD_CUDA_OK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  {
    // the coarse factorization is a chain of 128 small steps that shares the GPU
    // with the local factorization: its CTAs go first whenever an SM frees up
    int lo = 0, hi = 0;
    SFCDD_CUDA_OK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    SFCDD_CUDA_OK(cudaStreamCreateWithPriority(&h->side_stream, cudaStreamNonBlocking, hi));
  }
  cudaEvent_t e0, e1;
  SFCDD_CUDA_OK(cudaEventCreate(&e0));
  SFCDD_CUDA_OK(cudaEventCreate(&e1));
  SFCDD_CUDA_OK(cudaEventRecord(e0, h->stream));
  cudaStream_t s = h->stream;

  GridDev& g = h->g;

  // Algorithm 1, step 3: keys and curve order
  unsigned long long* keys;
  void* sort_tmp;
  TRY(dalloc(h, &keys, N));
  TRY(dalloc(h, &h->curve_code, N));
  TRY(dalloc(h, (unsigned char**)&sort_tmp, radix_sort_temp_bytes(h->N)));
  TRY(dalloc(h, &h->invpad, (size_t)1 << B));
  Prof pf(h, s);
  pf.run(SFCDD_K_KEYGEN, [&] { launch_keygen(g, keys, h->curve_code, s); });
  int sort_launches = 0;
  pf.run(SFCDD_K_SORT, [&] {
    radix_sort_pairs(keys, h->curve_code, h->N, d * nbits, sort_tmp, s, &sort_launches);
    cudaMemsetAsync(h->invpad, 0xff, ((size_t)1 << B) * sizeof(int), s);
    launch_invpad_fill(h->curve_code, h->invpad, h->N, s);
  });
  h->launches[SFCDD_K_SORT] += sort_launches;
  SFCDD_CUDA_OK(cudaGetLastError());

  // Algorithm 1, steps 4-5: partition, overlap, weights
  TRY(build_partition(h));
  TRY(dalloc(h, &h->d_start, P));
  TRY(dalloc(h, &h->d_len, P));
  TRY(dalloc(h, &h->d_omega, P));
  SFCDD_CUDA_OK(cudaMemcpyAsync(h->d_start, h->h_start.data(), P * sizeof(int), cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync(h->d_len, h->h_len.data(), P * sizeof(int), cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync(h->d_omega, h->h_omega.data(), P * sizeof(double), cudaMemcpyHostToDevice, s));
  PartDev& pd = h->pd;
  pd.N = h->N;
  pd.P = P;
  pd.q = h->q;
  pd.g = h->gfloor;
  pd.f = (int)(N / P);
  pd.r = (int)(N % P);
  pd.start = h->d_start;
  pd.len = h->d_len;
  pd.omega = h->d_omega;

  // tile layout: matrices 0..P-1 local, P coarse
  h->h_n.resize(P + 1);
  h->h_nt.resize(P + 1);
  h->h_tbase.resize(P + 1);
  h->h_vbase.resize(P + 1);
  long long vb = 0;
  h->max_nt = 0;
  int max_nlocal = 0;
  for (int m = 0; m <= P; ++m) {
    const int n = m < P ? h->h_len[m] : h->N0;
    const int nt = (n + TILE - 1) / TILE;
    h->h_n[m] = n;
    h->h_nt[m] = nt;
    h->h_vbase[m] = (int)vb;
    vb += (long long)nt * TILE;
    if (m < P) {
      h->max_nt = std::max(h->max_nt, nt);
      max_nlocal = std::max(max_nlocal, n);
    }
  }
  h->nt0 = h->h_nt[P];
  h->vtotal = vb;
  const int nrows = (int)(vb / TILE);  // tile rows over all matrices
  TRY(dalloc(h, &h->d_n, P + 1));
  TRY(dalloc(h, &h->d_nt, P + 1));
  TRY(dalloc(h, &h->d_tbase, P + 1));
  TRY(dalloc(h, &h->d_vbase, P + 1));
  TRY(dalloc(h, &h->d_zero64, 1));
  TRY(dalloc(h, &h->d_kmin, nrows));
  TRY(dalloc(h, &h->d_rowoff, nrows));
  TRY(dalloc(h, &h->d_colptr, nrows + 1));
  SFCDD_CUDA_OK(cudaMemsetAsync(h->d_zero64, 0, sizeof(long long), s));
  SFCDD_CUDA_OK(cudaMemcpyAsync(h->d_n, h->h_n.data(), (P + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync(h->d_nt, h->h_nt.data(), (P + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync(h->d_vbase, h->h_vbase.data(), (P + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  h->ts.nmat = P + 1;
  h->ts.n = h->d_n;
  h->ts.nt = h->d_nt;
  h->ts.tbase = h->d_tbase;
  h->ts.vbase = h->d_vbase;

  // Numbering of the coarse unknowns in the coarse factor: reverse
  // Cuthill-McKee on the graph of adjacent coarse blocks, a profile-reducing
  // order (A_0^{-1}, and so the coarse correction, is unchanged by it).  The
  // adjacency lists come from the device; the ordering is host bookkeeping on
  // N0 nodes, done while the device runs the local numbering below.
  int* d_adj = nullptr;
  int* d_deg = nullptr;
  std::vector<int> cdeg, cadj;
  int cdmax = 0;
  if (h->variant != SFCDD_ONE_LEVEL && h->N0 > 1) {
    const int N0 = h->N0;
    const int bmax = (pd.f + (pd.r > 0 ? 1 : 0) + h->q - 1) / h->q;
    const int maxdeg = std::min(N0 - 1, std::min(2048, std::max(32, bmax * 2 * d)));
    TRY(dalloc(h, &d_adj, (size_t)N0 * maxdeg));
    TRY(dalloc(h, &d_deg, N0));
    pf.run(SFCDD_K_COARSE_ASSEMBLE, [&] {
      launch_coarse_adjacency(g, pd, h->curve_code, h->invpad, maxdeg, d_adj, d_deg, s);
    });
    cdeg.resize(N0);
    SFCDD_CUDA_OK(cudaMemcpyAsync(cdeg.data(), d_deg, N0 * sizeof(int), cudaMemcpyDeviceToHost, s));
    SFCDD_CUDA_OK(cudaStreamSynchronize(s));
    bool ok = true;
    for (int v : cdeg) {
      if (v < 0) ok = false;
      cdmax = std::max(cdmax, v);
    }
    if (ok && cdmax > 0) {  // otherwise the coarse blocks keep the eq. restr order
      cadj.resize((size_t)N0 * cdmax);
      SFCDD_CUDA_OK(cudaMemcpy2DAsync(cadj.data(), cdmax * sizeof(int), d_adj, maxdeg * sizeof(int),
                                      cdmax * sizeof(int), N0, cudaMemcpyDeviceToHost, s));
      SFCDD_CUDA_OK(cudaStreamSynchronize(s));
    } else {
      cdmax = 0;
    }
  }

  // numbering inside each subdomain: lexicographic grid order by default (a
  // fill-reducing order; A_i^{-1} does not depend on it); queued here, waited
  // for after the coarse ordering
  h->local_order = o.local_order;
  std::vector<void*> order_tmp;
  std::vector<int> mstart, mN, mcb, lb;
  if (h->local_order == 0 && h->variant != SFCDD_COARSE_ONLY) {
    mstart.assign(P, 0);
    mN.assign(P, h->N);
    mcb.assign(P, 0);
    lb.assign(P, 0);
    long long tot = 0;
    for (int m = 0; m < P; ++m) {
      mstart[m] = h->h_start[m];
      lb[m] = (int)tot;
      tot += h->h_n[m];
    }
    int *d_ms, *d_mN, *d_mcb, *d_lb;
    unsigned long long* okeys;
    unsigned* ovals;
    unsigned char* otemp;
    TRY(dalloc(h, &d_ms, P));
    TRY(dalloc(h, &d_mN, P));
    TRY(dalloc(h, &d_mcb, P));
    TRY(dalloc(h, &d_lb, P));
    TRY(dalloc(h, &h->d_lperm, h->vtotal));
    TRY(dalloc(h, &h->d_linv, h->vtotal));
    TRY(dalloc(h, &okeys, tot));
    TRY(dalloc(h, &ovals, tot));
    TRY(dalloc(h, &otemp, radix_sort_temp_bytes((int)tot)));
    SFCDD_CUDA_OK(cudaMemcpyAsync(d_ms, mstart.data(), P * sizeof(int), cudaMemcpyHostToDevice, s));
    SFCDD_CUDA_OK(cudaMemcpyAsync(d_mN, mN.data(), P * sizeof(int), cudaMemcpyHostToDevice, s));
    SFCDD_CUDA_OK(cudaMemcpyAsync(d_mcb, mcb.data(), P * sizeof(int), cudaMemcpyHostToDevice, s));
    SFCDD_CUDA_OK(cudaMemcpyAsync(d_lb, lb.data(), P * sizeof(int), cudaMemcpyHostToDevice, s));
    pf.run(SFCDD_K_SORT, [&] {
      local_order_lex(h->ts, P, max_nlocal, d_ms, d_mN, d_mcb, d_lb, tot, h->curve_code, okeys,
                      ovals, otemp, h->d_lperm, h->d_linv, s);
    });
    order_tmp = {(void*)okeys, (void*)ovals, (void*)otemp, (void*)d_ms,
                 (void*)d_mN,  (void*)d_mcb, (void*)d_lb};
    h->ts.lperm = h->d_lperm;
    h->ts.linv = h->d_linv;
  }

  std::vector<int> corder, crow;
  if (cdmax > 0) {
    const int N0 = h->N0;
    rcm_order(N0, cdeg, cadj, cdmax, corder);
    crow.resize(N0);
    for (int r = 0; r < N0; ++r) crow[corder[r]] = r;
    TRY(dalloc(h, &h->d_crow, N0));
    TRY(dalloc(h, &h->d_cblock, N0));
    SFCDD_CUDA_OK(cudaMemcpyAsync(h->d_crow, crow.data(), N0 * sizeof(int), cudaMemcpyHostToDevice, s));
    SFCDD_CUDA_OK(cudaMemcpyAsync(h->d_cblock, corder.data(), N0 * sizeof(int), cudaMemcpyHostToDevice, s));
    pd.crow = h->d_crow;
    pd.cblock = h->d_cblock;
  }
  SFCDD_CUDA_OK(cudaStreamSynchronize(s));  // host vectors above go out of scope
  for (void* t : order_tmp) dfree(h, t);
  dfree(h, d_adj);
  dfree(h, d_deg);

  // Cholesky envelopes of every local matrix and of the coarse matrix: the
  // first column with a nonzero in each tile row (the factor keeps that profile)
  SkylineHost sky;
  {
    const int max_nt_all = std::max(h->max_nt, h->nt0);
    int* tfirst = nullptr;
    TRY(dalloc(h, &tfirst, nrows));
    pf.run(SFCDD_K_ASSEMBLE, [&] {
      launch_envelope_init(h->ts, P + 1, max_nt_all, tfirst, s);
      if (h->variant != SFCDD_COARSE_ONLY)
        launch_envelope_local(g, pd, h->curve_code, h->invpad, h->ts, P, max_nlocal, tfirst, s);
      if (h->variant != SFCDD_ONE_LEVEL)
        launch_envelope_coarse(g, pd, h->curve_code, h->invpad, h->h_vbase[P] / TILE, tfirst, s);
    });
    std::vector<int> tf(nrows);
    SFCDD_CUDA_OK(cudaMemcpyAsync(tf.data(), tfirst, nrows * sizeof(int), cudaMemcpyDeviceToHost, s));
    SFCDD_CUDA_OK(cudaStreamSynchronize(s));
    dfree(h, tfirst);
    std::vector<char> is_coarse(P + 1, 0);
    is_coarse[P] = 1;
    std::vector<int> cb(P + 1, 1);
    cb[P] = h->cb_coarse;
    build_skyline(h->h_nt, h->h_vbase, is_coarse, cb, tf, sky);
  }
  h->h_kmin = sky.kmin;
  h->h_rowoff = sky.rowoff;
  h->stored = sky.stored;
  for (int m = 0; m <= P; ++m) h->h_tbase[m] = sky.tbase[m];
  h->max_ltiles = sky.max_ltiles;
  h->max_ctiles = sky.max_ctiles;
  h->fwd_tiles_l = sky.fwd_tiles_l;
  h->bwd_tiles_l = sky.bwd_tiles_l;
  h->fwd_tiles_c = sky.fwd_tiles_c;
  h->bwd_tiles_c = sky.bwd_tiles_c;
  h->ltile_elems = sky.ltiles * TILE2;
  h->ctile_elems = sky.ctiles * TILE2;
  h->col_max_local = sky.col_max_local;
  h->col_max_coarse = sky.col_max_coarse;
  if (h->variant != SFCDD_COARSE_ONLY) {
    h->work_potrf = sky.potrf;
    h->work_trsm = sky.trsm;
    h->work_syrk = sky.syrk;
  }
  if (h->variant != SFCDD_ONE_LEVEL) h->work_coarse = sky.coarse;
  h->factor_flops = h->work_potrf + h->work_trsm + h->work_syrk;
  std::vector<int>& colptr = sky.colptr;
  std::vector<int>& colidx = sky.colidx;
  TRY(dalloc(h, &h->d_colidx, colidx.size()));
  SFCDD_CUDA_OK(cudaMemcpyAsync(h->d_kmin, h->h_kmin.data(), nrows * sizeof(int), cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync(h->d_rowoff, h->h_rowoff.data(), nrows * sizeof(int), cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync(h->d_colptr, colptr.data(), (nrows + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync(h->d_colidx, colidx.data(), colidx.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync(h->d_tbase, h->h_tbase.data(), (P + 1) * sizeof(long long), cudaMemcpyHostToDevice, s));
  h->ts.kmin = h->d_kmin;
  h->ts.rowoff = h->d_rowoff;
  h->ts.colptr = h->d_colptr;
  h->ts.colidx = h->d_colidx;
  // zero-row bounds: whole tiles until the local factors are scanned
  h->h_nzr.assign(nrows, TILE);
  TRY(dalloc(h, &h->d_nzr, nrows));
  SFCDD_CUDA_OK(cudaMemcpyAsync(h->d_nzr, h->h_nzr.data(), nrows * sizeof(int), cudaMemcpyHostToDevice, s));
  h->ts.nzr = h->d_nzr;
  SFCDD_CUDA_OK(cudaStreamSynchronize(s));  // host vectors above go out of scope

  TRY(dalloc(h, &h->err, 1));
  SFCDD_CUDA_OK(cudaMemsetAsync(h->err, 0, sizeof(ErrWord), s));
  int* diag_cnt = nullptr;  // per tile row: updates of its diagonal tile seen (factorization)
  TRY(dalloc(h, &diag_cnt, nrows));
  SFCDD_CUDA_OK(cudaMemsetAsync(diag_cnt, 0, nrows * sizeof(int), s));

  // Algorithm 1, steps 9-10: coarse matrix and its FP64 factor, on a side
  // stream so that it overlaps the local factorization (the two are independent)
  TRY(dalloc(h, &h->ctiles, h->ctile_elems));
  TRY(dalloc(h, &h->cut, h->ctile_elems));
  double* xs = nullptr;  // inverses of the coarse diagonal blocks (scratch)
  const int cnblk = (h->nt0 + h->cb_coarse - 1) / h->cb_coarse;
  if (h->cb_coarse > 1)
    TRY(dalloc(h, &xs, (size_t)cnblk * h->cb_coarse * h->cb_coarse * TILE2));
  cudaEvent_t ev_fork = nullptr, ev_coarse = nullptr;
  SFCDD_CUDA_OK(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
  SFCDD_CUDA_OK(cudaEventCreateWithFlags(&ev_coarse, cudaEventDisableTiming));
  SFCDD_CUDA_OK(cudaEventRecord(ev_fork, s));
  SFCDD_CUDA_OK(cudaStreamWaitEvent(h->side_stream, ev_fork, 0));
  cudaEventDestroy(ev_fork);
  Prof pf2(h, h->side_stream);
  if (h->variant != SFCDD_ONE_LEVEL) {
    cudaStream_t s2 = h->side_stream;
    // the coarse matrix is a one-matrix tile set with base 0
    const TileSetDev cts = coarse_view(h);
    pf2.run(SFCDD_K_COARSE_ASSEMBLE, [&] {
      launch_assemble_coarse(g, pd, h->curve_code, h->invpad, cts, h->stored[P], h->ctiles, s2);
    });
    CoarseHook ch(pf2);
    factor_tiles(cts, 0, 1, h->nt0, h->col_max_coarse.data(), h->ctiles, Store::F64, diag_cnt,
                 h->err, s2, &ch, 4, h->tensor_cores);
    pf2.run(SFCDD_K_COARSE_FACTOR, [&] {
      if (h->cb_coarse > 1)
        unitize_blocks(cts, h->nt0, h->cb_coarse, h->stored[P], h->ctiles, h->cut, xs, s2);
      else
        unitize_tiles(cts, 0, 1, h->max_ctiles, h->ctiles, h->cut, Store::F64, s2);
    });
  }
  SFCDD_CUDA_OK(cudaEventRecord(ev_coarse, h->side_stream));

  // Algorithm 1, steps 6-7 and Sec. 3.1: local matrices and their factors
  const Store compute_st = h->st == Store::BF16 ? Store::F32 : h->st;
  const size_t esz = compute_st == Store::F64 ? 8 : 4;
  if (h->variant == SFCDD_COARSE_ONLY) h->ltile_elems = 0;  // no local problems
  void* work_tiles = nullptr;
  TRY(dalloc(h, (unsigned char**)&work_tiles, h->ltile_elems * esz));
  if (h->variant != SFCDD_COARSE_ONLY) {
    pf.run(SFCDD_K_ASSEMBLE, [&] {
      launch_assemble_local(g, pd, h->curve_code, h->invpad, h->ts, 0, P, h->max_ltiles,
                            work_tiles, compute_st, s);
    });
    factor_tiles(h->ts, 0, P, h->max_nt, h->col_max_local.data(), work_tiles, compute_st, diag_cnt,
                 h->err, s, &pf, compute_st == Store::F64 ? 4 : 1, h->tensor_cores,
                 h->bf16_operands);
  }
  // substitution form: Lh in place, Lh^T and E_K into a second tile array
  NvtxRange nvtx_unit("sfcdd setup: substitution form");
  void* work_ut = nullptr;
  TRY(dalloc(h, (unsigned char**)&work_ut, h->ltile_elems * esz));
  if (h->variant != SFCDD_COARSE_ONLY)
    pf.run(SFCDD_K_TRSM, [&] {
      unitize_tiles(h->ts, 0, P, h->max_ltiles, work_tiles, work_ut, compute_st, s);
    });
  if (h->st == Store::BF16) {
    TRY(dalloc(h, (__nv_bfloat16**)&h->ltiles, h->ltile_elems));
    TRY(dalloc(h, (__nv_bfloat16**)&h->lut, h->ltile_elems));
    pf.run(SFCDD_K_VECTOR, [&] {
      launch_convert_f32_bf16((const float*)work_tiles, (__nv_bfloat16*)h->ltiles, h->ltile_elems, s);
      launch_convert_f32_bf16((const float*)work_ut, (__nv_bfloat16*)h->lut, h->ltile_elems, s);
    });
    SFCDD_CUDA_OK(cudaStreamSynchronize(s));
    dfree(h, work_tiles);
    dfree(h, work_ut);
  } else {
    h->ltiles = work_tiles;
    h->lut = work_ut;
  }
  if (h->variant != SFCDD_COARSE_ONLY)
    pf.run(SFCDD_K_TRSM, [&] {
      launch_offblock_rows(h->ts, 0, P, h->max_nt, h->ltiles, h->st, h->d_nzr, s);
      if (h->st == Store::F64)
        launch_pack_half_tiles(h->ts, 0, P, h->max_ltiles, (double*)h->lut, h->d_nzr, s);
    });
  SFCDD_CUDA_OK(cudaGetLastError());

  // The host bookkeeping below (work lists, solve buffers) waits for the local
  // work on s only; the coarse factorization, usually the longer of the two,
  // keeps running on the side stream and is joined just before the end event.
  if (h->auto_local && h->variant != SFCDD_COARSE_ONLY && whole_fits(h->st, h->max_nt))
    h->nsub_local = 0;
  TRY(configure_substitution(h, h->nsub_local, h->nsub_coarse));
  if (h->variant == SFCDD_BALANCED)
    for (int k = 0; k < 4; ++k) TRY(dalloc(h, &h->bal[k], N));
  TRY(dalloc(h, &h->ybuf, h->vtotal));
  TRY(dalloc(h, &h->dbuf, h->vtotal));
  TRY(dalloc(h, &h->zcbuf, h->vtotal));
  launch_fill_pending(h->ybuf, h->vtotal, s);
  launch_fill_pending(h->dbuf, h->vtotal, s);

  // PCG state
  TRY(dalloc(h, &h->b, N));
  TRY(dalloc(h, &h->x, N));
  TRY(dalloc(h, &h->r, N));
  TRY(dalloc(h, &h->p, N));
  TRY(dalloc(h, &h->qv, N));
  TRY(dalloc(h, &h->z, N));
  TRY(dalloc(h, &h->tmp, N));
  TRY(dalloc(h, &h->tmp2, N));
  TRY(dalloc(h, &h->g0, (size_t)h->nt0 * TILE));
  SFCDD_CUDA_OK(cudaMemsetAsync(h->g0, 0, (size_t)h->nt0 * TILE * sizeof(double), s));
  TRY(dalloc(h, &h->sc, 1));
  SFCDD_CUDA_OK(cudaMemsetAsync(h->sc, 0, sizeof(PcgScalars), s));
  SFCDD_CUDA_OK(cudaMallocHost((void**)&h->sc_host, sizeof(PcgScalars)));
  h->ws.nblocks = vec_blocks(h->N);
  TRY(dalloc(h, &h->ws.partial, (size_t)h->ws.nblocks * MAXD));
  TRY(dalloc(h, &h->ws.counter, 1));
  SFCDD_CUDA_OK(cudaMemsetAsync(h->ws.counter, 0, sizeof(unsigned), s));
  if (h->variant != SFCDD_BALANCED) TRY(setup_fused(h));

  SFCDD_CUDA_OK(cudaStreamWaitEvent(s, ev_coarse, 0));
  cudaEventDestroy(ev_coarse);
  SFCDD_CUDA_OK(cudaEventRecord(e1, s));
  SFCDD_CUDA_OK(cudaEventSynchronize(e1));
  pf.collect();
  pf2.collect();
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  h->setup_ms = ms;
  TRY(count_local_elems(h));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (xs) dfree(h, xs);
  dfree(h, diag_cnt);
  dfree(h, keys);
  dfree(h, sort_tmp);
  int fi = 0;
  const int ec = check_err(h, &fi);
  if (ec != 0) return ec;
  return SFCDD_OK;
}

void destroy_impl(sfcdd_handle* h) {
  if (!h) return;
  if (h->iter_graph) cudaGraphExecDestroy(h->iter_graph);
  for (void* p : h->allocs)
    if (p) cudaFree(p);
  if (h->sc_host) cudaFreeHost(h->sc_host);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->side_stream) cudaStreamDestroy(h->side_stream);
  delete h;
}

int read_scalars(sfcdd_handle* h) {
  SFCDD_CUDA_OK(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, h->stream));
  SFCDD_CUDA_OK(cudaStreamSynchronize(h->stream));
  return SFCDD_OK;
}

// PCG on the curve-order right-hand side already in h->b; solution in h->x.
// homogeneous: b = 0 and h->x holds x_0; the iteration stops on the energy
// norm ||x_k||_A <= rtol ||x_0||_A (Sec. 4) instead of the residual.
int pcg_impl(sfcdd_handle* h, double rtol, int maxit, sfcdd_stats* stats,
             bool homogeneous = false) {
  NvtxRange nvtx("sfcdd pcg");
  if (!(rtol >= 0) || maxit < 0) return SFCDD_ERR_INVALID_ARG;
  cudaStream_t s = h->stream;
  TRY(build_graph(h));
  cudaEvent_t e0, e1;
  SFCDD_CUDA_OK(cudaEventCreate(&e0));
  SFCDD_CUDA_OK(cudaEventCreate(&e1));
  SFCDD_CUDA_OK(cudaEventRecord(e0, s));
  Prof pf(h, s);
  if (homogeneous) {
    // r_0 = -A x_0, ||x_0||_A^2 = -x_0^T r_0
    pf.run(SFCDD_K_STENCIL, [&] {
      launch_residual(h->g, h->curve_code, h->invpad, h->b, h->x, h->r, nullptr, h->ws, s);
    });
    pf.run(SFCDD_K_VECTOR, [&] {
      launch_energy(h->N, h->x, h->r, h->sc, h->ws, rtol, h->flexible, 1, s);
    });
  } else {
    pf.run(SFCDD_K_VECTOR, [&] { launch_init_pcg(h->N, h->b, h->x, h->r, h->sc, h->ws, rtol, h->flexible, s); });
  }
  SFCDD_CUDA_OK(cudaMemsetAsync(h->p, 0, (size_t)h->N * sizeof(double), s));
  SFCDD_CUDA_OK(cudaMemsetAsync(h->z, 0, (size_t)h->N * sizeof(double), s));
  if (h->fused) {
    // every iteration is {substitutions, vector phase}: the first needs R_0 r_0;
    // the vector phase's barrier counts arrivals from the start of the solve
    SFCDD_CUDA_OK(cudaMemsetAsync(h->p2, 0, (size_t)h->N * sizeof(double), s));
    SFCDD_CUDA_OK(cudaMemsetAsync(h->fz.bar, 0, 2 * sizeof(unsigned), s));
    if (h->variant != SFCDD_ONE_LEVEL)
      pf.run(SFCDD_K_RESTRICT, [&] { launch_restrict(h->pd, h->r, h->g0, h->sc, s); });
  } else {
    enqueue_apply(h, pf, h->r, h->z, h->sc);   // z_0 = C^{-1} r_0, rz, beta = 0
    pf.run(SFCDD_K_VECTOR, [&] { launch_update_p(h->N, h->z, h->p, h->sc, s); });
  }
  int launched = 0;
  int chunk = 2;
  int rc = SFCDD_OK;
  while (true) {
    TRY(read_scalars(h));
    if (h->sc_host->done || h->sc_host->status) break;
    if (launched >= maxit) break;
    const int n = std::min(chunk, maxit - launched);
    for (int k = 0; k < n; ++k) {
      if (h->profiling) {
        enqueue_iteration(h, pf);
        if (h->fused_rc) return h->fused_rc;
      } else {
        SFCDD_CUDA_OK(cudaGraphLaunch(h->iter_graph, s));
        for (int c = 0; c < SFCDD_K_COUNT; ++c) h->launches[c] += h->graph_kernels[c];
      }
    }
    launched += n;
    chunk = std::min(chunk * 2, 16);
  }
  SFCDD_CUDA_OK(cudaEventRecord(e1, s));
  if (homogeneous) {
    // energy norm recomputed from A x (not the recurrence residual)
    pf.run(SFCDD_K_STENCIL, [&] {
      launch_residual(h->g, h->curve_code, h->invpad, h->b, h->x, h->tmp, nullptr, h->ws, s);
    });
    pf.run(SFCDD_K_VECTOR,
           [&] { launch_energy(h->N, h->x, h->tmp, h->sc, h->ws, rtol, h->flexible, 0, s); });
  } else {
    // true residual ||b - A x|| / ||b||
    pf.run(SFCDD_K_STENCIL, [&] {
      launch_true_residual(h->g, h->curve_code, h->invpad, h->b, h->x, h->tmp, h->sc, h->ws, s);
    });
  }
  TRY(read_scalars(h));
  pf.collect();
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->solve_ms = ms;
  int fi = 0;
  const int ec = check_err(h, &fi);
  const PcgScalars& sc = *h->sc_host;
  if (ec != 0) rc = ec;
  else if (sc.status) rc = sc.status;
  else if (!sc.done) rc = SFCDD_ERR_MAXIT;
  if (stats) {
    stats->iters = sc.iter;
    stats->status = rc;
    stats->fail_index = fi;
    stats->rel_res = sc.rel;
    stats->true_rel_res = sc.true_rel;
    stats->setup_ms = h->setup_ms;
    stats->solve_ms = ms;
  }
  return rc;
}

// Algorithm 3 on the curve-order right-hand side in h->b: x <- x + xi C^{-1}(b - A x),
// result written to u_dev (lexicographic).  homogeneous: b = 0, h->x holds x_0 and
// the stop is ||x_k||_A <= rtol ||x_0||_A (Sec. 4); otherwise x_0 = 0 and the stop
// is the true relative residual.  Every step reads the stopping quantity back.
int richardson_impl(sfcdd_handle* h, double* u_dev, double xi, double rtol, int maxit,
                    sfcdd_stats* stats, bool homogeneous) {
  NvtxRange nvtx("sfcdd richardson");
  cudaStream_t s = h->stream;
  cudaEvent_t e0, e1;
  SFCDD_CUDA_OK(cudaEventCreate(&e0));
  SFCDD_CUDA_OK(cudaEventCreate(&e1));
  SFCDD_CUDA_OK(cudaEventRecord(e0, s));
  Prof pf(h, s);
  if (!homogeneous)
    pf.run(SFCDD_K_VECTOR,
           [&] { launch_init_pcg(h->N, h->b, h->x, h->r, h->sc, h->ws, rtol, 0, s); });
  int k = 0;
  int rc = SFCDD_OK;
  for (;;) {
    if (homogeneous) {
      // tmp = -A x; ||x||_A^2 = -x^T tmp (the first pass records ||x_0||_A)
      pf.run(SFCDD_K_STENCIL, [&] {
        launch_residual(h->g, h->curve_code, h->invpad, h->b, h->x, h->tmp, nullptr, h->ws, s);
      });
      pf.run(SFCDD_K_VECTOR,
             [&] { launch_energy(h->N, h->x, h->tmp, h->sc, h->ws, rtol, 0, k == 0, s); });
    } else {
      // tmp = b - A x and ||tmp|| / ||b||
      pf.run(SFCDD_K_STENCIL, [&] {
        launch_true_residual(h->g, h->curve_code, h->invpad, h->b, h->x, h->tmp, h->sc, h->ws, s);
      });
    }
    TRY(read_scalars(h));
    if (h->sc_host->status) {  // non-finite input seen by the initialization
      rc = h->sc_host->status;
      break;
    }
    const double rel = (homogeneous || h->sc_host->bb > 0) ? h->sc_host->true_rel : 0.0;
    if (!(rel == rel)) {
      rc = SFCDD_ERR_NAN;
      break;
    }
    if (rel <= rtol) break;
    if (k >= maxit) {
      rc = SFCDD_ERR_MAXIT;
      break;
    }
    enqueue_apply(h, pf, h->tmp, h->z, nullptr);  // z = C^{-1} (b - A x)
    pf.run(SFCDD_K_UPDATE, [&] { launch_axpby(h->N, 1.0, h->x, xi, h->z, h->x, s); });
    ++k;
  }
  SFCDD_CUDA_OK(cudaEventRecord(e1, s));
  SFCDD_CUDA_OK(cudaEventSynchronize(e1));
  pf.collect();
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int fi = 0;
  const int ec = check_err(h, &fi);
  if (ec != 0) rc = ec;
  h->launches[SFCDD_K_VECTOR] += 1;
  launch_curve_to_lex(h->g, h->curve_code, h->x, u_dev, s);
  SFCDD_CUDA_OK(cudaStreamSynchronize(s));
  if (stats) {
    stats->iters = k;
    stats->status = rc;
    stats->fail_index = fi;
    stats->rel_res = h->sc_host->true_rel;
    stats->true_rel_res = h->sc_host->true_rel;
    stats->setup_ms = h->setup_ms;
    stats->solve_ms = ms;
  }
  return rc;
}

}  // namespace

// ===========================================================================
extern "C" {

void sfcdd_default_options(sfcdd_options* opt) {
  if (!opt) return;
  opt->coeffs = nullptr;
  opt->q = 0;
  opt->variant = SFCDD_ADDITIVE;
  opt->weighting = SFCDD_WEIGHT_OMEGA;
  opt->precision = SFCDD_FP64;
  opt->flexible = -1;
  opt->stream = nullptr;
  opt->profile = 0;
  opt->local_order = 0;
  opt->slabs_local = 0;
  opt->slabs_coarse = 0;
  opt->tensor_cores = -1;
}

int sfcdd_setup_ex(const int* levels, int d, int P, double overlap, const sfcdd_options* opt,
                   sfcdd_handle** out) {
  if (!out) return SFCDD_ERR_INVALID_ARG;
  *out = nullptr;
  sfcdd_handle* h = new (std::nothrow) sfcdd_handle();
  if (!h) return SFCDD_ERR_NOMEM;
  const int rc = setup_impl(h, levels, d, P, overlap, opt);
  if (rc != SFCDD_OK) {
    if (h->stream) cudaStreamSynchronize(h->stream);
    destroy_impl(h);
    return rc;
  }
  *out = h;
  return SFCDD_OK;
}

int sfcdd_setup(const int* levels, int d, int P, double overlap, sfcdd_handle** out) {
  return sfcdd_setup_ex(levels, d, P, overlap, nullptr, out);
}

int sfcdd_solve(sfcdd_handle* h, const double* f_dev, double* u_dev, double rtol, int maxit,
                sfcdd_stats* stats) {
  if (!h || !f_dev || !u_dev) return SFCDD_ERR_INVALID_ARG;
  cudaStream_t s = h->stream;
  h->launches[SFCDD_K_VECTOR] += 1;
  launch_lex_to_curve(h->g, h->curve_code, f_dev, h->b, s);
  const int rc = pcg_impl(h, rtol, maxit, stats);
  if (rc == SFCDD_OK || rc == SFCDD_ERR_MAXIT) {
    h->launches[SFCDD_K_VECTOR] += 1;
    launch_curve_to_lex(h->g, h->curve_code, h->x, u_dev, s);
    SFCDD_CUDA_OK(cudaStreamSynchronize(s));
  }
  return rc;
}

int sfcdd_solve_host(sfcdd_handle* h, const double* f_host, double* u_host, double rtol, int maxit,
                     sfcdd_stats* stats) {
  if (!h || !f_host || !u_host) return SFCDD_ERR_INVALID_ARG;
  cudaStream_t s = h->stream;
  SFCDD_CUDA_OK(cudaMemcpyAsync(h->tmp2, f_host, (size_t)h->N * sizeof(double), cudaMemcpyHostToDevice, s));
  h->launches[SFCDD_K_VECTOR] += 1;
  launch_lex_to_curve(h->g, h->curve_code, h->tmp2, h->b, s);
  const int rc = pcg_impl(h, rtol, maxit, stats);
  if (rc == SFCDD_OK || rc == SFCDD_ERR_MAXIT) {
    h->launches[SFCDD_K_VECTOR] += 1;
    launch_curve_to_lex(h->g, h->curve_code, h->x, h->tmp2, s);
    SFCDD_CUDA_OK(cudaMemcpyAsync(u_host, h->tmp2, (size_t)h->N * sizeof(double), cudaMemcpyDeviceToHost, s));
    SFCDD_CUDA_OK(cudaStreamSynchronize(s));
  }
  return rc;
}

int sfcdd_solve_backward(sfcdd_handle* h, const double* u_dev, const double* gu_dev, double* gf_dev,
                         double* gc_host, double rtol, int maxit, sfcdd_stats* stats) {
  if (!h || !u_dev || !gu_dev) return SFCDD_ERR_INVALID_ARG;
  cudaStream_t s = h->stream;
  h->launches[SFCDD_K_VECTOR] += 1;
  launch_lex_to_curve(h->g, h->curve_code, gu_dev, h->b, s);
  const int rc = pcg_impl(h, rtol, maxit, stats);   // x = lambda (curve order)
  if (rc != SFCDD_OK && rc != SFCDD_ERR_MAXIT) return rc;
  if (gf_dev) {
    h->launches[SFCDD_K_VECTOR] += 1;
    launch_curve_to_lex(h->g, h->curve_code, h->x, gf_dev, s);
  }
  if (gc_host) {
    h->launches[SFCDD_K_VECTOR] += 1;
    launch_lex_to_curve(h->g, h->curve_code, u_dev, h->tmp, s);
    h->launches[SFCDD_K_GRAD] += 1;
    launch_grad(h->g, h->curve_code, h->invpad, h->x, h->tmp, h->sc, h->ws, s);
    TRY(read_scalars(h));
    for (int j = 0; j < h->d; ++j) gc_host[j] = h->sc_host->grad[j];
  }
  SFCDD_CUDA_OK(cudaStreamSynchronize(s));
  return rc;
}

namespace {
// Number of eigenvalues below x of the symmetric tridiagonal (d, e), e[j]
// coupling j-1 and j (Sturm sequence of the LDL^T pivots).
int sturm_count(const std::vector<double>& d, const std::vector<double>& e, double x) {
  int cnt = 0;
  double q = 1.0;
  for (size_t j = 0; j < d.size(); ++j) {
    const double off = j ? e[j] * e[j] / q : 0.0;
    q = d[j] - x - off;
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}
// The idx-th smallest eigenvalue by bisection inside the Gershgorin interval.
double tridiag_eig(const std::vector<double>& d, const std::vector<double>& e, int idx) {
  double lo = 1e300, hi = -1e300;
  for (size_t j = 0; j < d.size(); ++j) {
    const double r = (j ? std::fabs(e[j]) : 0.0) + (j + 1 < d.size() ? std::fabs(e[j + 1]) : 0.0);
    lo = std::min(lo, d[j] - r);
    hi = std::max(hi, d[j] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_count(d, e, mid) > idx) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}
}  // namespace

int sfcdd_estimate_spectrum(sfcdd_handle* h, const double* f_dev, int steps, double* lmin,
                            double* lmax) {
  if (!h || !f_dev || steps < 1 || !lmin || !lmax) return SFCDD_ERR_INVALID_ARG;
  cudaStream_t s = h->stream;
  double* hist = nullptr;
  SFCDD_CUDA_OK(cudaMalloc(&hist, 2 * (size_t)steps * sizeof(double)));
  double* ha = hist;
  double* hb = hist + steps;
  const PcgScalars* sc = h->sc;
  SFCDD_CUDA_OK(cudaMemcpyAsync((char*)h->sc + offsetof(PcgScalars, hist_alpha), &ha, sizeof(ha),
                                cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync((char*)h->sc + offsetof(PcgScalars, hist_beta), &hb, sizeof(hb),
                                cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync((char*)h->sc + offsetof(PcgScalars, hist_cap), &steps, sizeof(int),
                                cudaMemcpyHostToDevice, s));
  (void)sc;
  h->launches[SFCDD_K_VECTOR] += 1;
  launch_lex_to_curve(h->g, h->curve_code, f_dev, h->b, s);
  sfcdd_stats st{};
  int rc = pcg_impl(h, 1e-14, steps, &st);
  std::vector<double> a(steps), b(steps);
  SFCDD_CUDA_OK(cudaMemcpyAsync(a.data(), ha, steps * sizeof(double), cudaMemcpyDeviceToHost, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync(b.data(), hb, steps * sizeof(double), cudaMemcpyDeviceToHost, s));
  const double* nul = nullptr;
  const int zero = 0;
  SFCDD_CUDA_OK(cudaMemcpyAsync((char*)h->sc + offsetof(PcgScalars, hist_alpha), &nul, sizeof(nul),
                                cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync((char*)h->sc + offsetof(PcgScalars, hist_beta), &nul, sizeof(nul),
                                cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaMemcpyAsync((char*)h->sc + offsetof(PcgScalars, hist_cap), &zero, sizeof(int),
                                cudaMemcpyHostToDevice, s));
  SFCDD_CUDA_OK(cudaStreamSynchronize(s));
  cudaFree(hist);
  if (rc != SFCDD_OK && rc != SFCDD_ERR_MAXIT) return rc;
  const int k = std::min(st.iters, steps);
  if (k < 1) return SFCDD_ERR_INVALID_ARG;
  // Lanczos tridiagonal of C^{-1} A from the PCG coefficients:
  // T_00 = 1/a_0, T_jj = 1/a_j + b_{j-1}/a_{j-1}, T_{j-1,j} = sqrt(b_{j-1})/a_{j-1}
  std::vector<double> d(k), e(k, 0.0);
  for (int j = 0; j < k; ++j) {
    d[j] = 1.0 / a[j] + (j ? b[j - 1] / a[j - 1] : 0.0);
    if (j) e[j] = std::sqrt(std::max(b[j - 1], 0.0)) / a[j - 1];
  }
  *lmin = tridiag_eig(d, e, 0);
  *lmax = tridiag_eig(d, e, k - 1);
  return SFCDD_OK;
}

int sfcdd_richardson(sfcdd_handle* h, const double* f_dev, double* u_dev, double xi, double rtol,
                     int maxit, sfcdd_stats* stats) {
  if (!h || !f_dev || !u_dev || !(xi > 0) || !(rtol >= 0) || maxit < 0)
    return SFCDD_ERR_INVALID_ARG;
  h->launches[SFCDD_K_VECTOR] += 1;
  launch_lex_to_curve(h->g, h->curve_code, f_dev, h->b, h->stream);
  return richardson_impl(h, u_dev, xi, rtol, maxit, stats, false);
}

int sfcdd_solve_homogeneous(sfcdd_handle* h, const double* x0_dev, double* u_dev, int method,
                            double xi, double tol, int maxit, sfcdd_stats* stats) {
  if (!h || !x0_dev || !u_dev || !(tol >= 0) || maxit < 0) return SFCDD_ERR_INVALID_ARG;
  if (method != SFCDD_METHOD_PCG && method != SFCDD_METHOD_RICHARDSON)
    return SFCDD_ERR_INVALID_ARG;
  if (method == SFCDD_METHOD_RICHARDSON && !(xi > 0)) return SFCDD_ERR_INVALID_ARG;
  cudaStream_t s = h->stream;
  SFCDD_CUDA_OK(cudaMemsetAsync(h->b, 0, (size_t)h->N * sizeof(double), s));
  h->launches[SFCDD_K_VECTOR] += 1;
  launch_lex_to_curve(h->g, h->curve_code, x0_dev, h->x, s);
  if (method == SFCDD_METHOD_RICHARDSON)
    return richardson_impl(h, u_dev, xi, tol, maxit, stats, true);
  const int rc = pcg_impl(h, tol, maxit, stats, true);
  h->launches[SFCDD_K_VECTOR] += 1;
  launch_curve_to_lex(h->g, h->curve_code, h->x, u_dev, s);
  SFCDD_CUDA_OK(cudaStreamSynchronize(s));
  return rc;
}

int sfcdd_apply_operator(sfcdd_handle* h, const double* x_dev, double* y_dev, int curve_order) {
  if (!h || !x_dev || !y_dev) return SFCDD_ERR_INVALID_ARG;
  cudaStream_t s = h->stream;
  Prof pf(h, s);
  if (curve_order) {
    pf.run(SFCDD_K_STENCIL, [&] { launch_stencil(h->g, h->curve_code, h->invpad, x_dev, y_dev, 0, nullptr, h->ws, s); });
  } else {
    h->launches[SFCDD_K_VECTOR] += 2;
    launch_lex_to_curve(h->g, h->curve_code, x_dev, h->tmp, s);
    pf.run(SFCDD_K_STENCIL, [&] { launch_stencil(h->g, h->curve_code, h->invpad, h->tmp, h->tmp2, 0, nullptr, h->ws, s); });
    launch_curve_to_lex(h->g, h->curve_code, h->tmp2, y_dev, s);
  }
  SFCDD_CUDA_OK(cudaGetLastError());
  pf.collect();
  return SFCDD_OK;
}

int sfcdd_selftest(sfcdd_handle* h, int kind, int* detail) {
  if (!h || (kind != SFCDD_SELFTEST_WAIT_TIMEOUT && kind != SFCDD_SELFTEST_BREAKDOWN))
    return SFCDD_ERR_INVALID_ARG;
  cudaStream_t s = h->stream;
  SFCDD_CUDA_OK(cudaStreamSynchronize(s));
  SFCDD_CUDA_OK(cudaMemsetAsync(h->err, 0, sizeof(ErrWord), s));
  if (kind == SFCDD_SELFTEST_BREAKDOWN) {
    // identity with a negative pivot at row 17: the diagonal factorization must
    // report NOT_SPD with the index it was given
    std::vector<double> a(TILE2, 0.0);
    for (int i = 0; i < TILE; ++i) a[(size_t)i * TILE + i] = i == 17 ? -1.0 : 2.0;
    double* t = nullptr;
    SFCDD_CUDA_OK(cudaMalloc(&t, TILE2 * sizeof(double)));
    SFCDD_CUDA_OK(cudaMemcpyAsync(t, a.data(), TILE2 * sizeof(double), cudaMemcpyHostToDevice, s));
    launch_potrf_one(t, h->err, 4242, s);
    SFCDD_CUDA_OK(cudaStreamSynchronize(s));
    cudaFree(t);
  } else {
    // a forward substitution whose first work item never runs: the items that
    // depend on its rows wait on result slots nothing writes, give up after the
    // bounded spin, record TIMEOUT, and every other waiter then stops waiting.
    // Whole-matrix items depend on nothing, so the test runs on row slabs.
    const int keep_l = h->nsub_local;
    if (keep_l == 0) TRY(configure_substitution(h, 1, h->nsub_coarse));
    const auto& wl = h->lists[LIST_MAIN];
    if (wl.n < 2) return SFCDD_ERR_INVALID_ARG;
    const unsigned long long one = 1;
    SFCDD_CUDA_OK(cudaMemcpyAsync(wl.tf, &one, sizeof(one), cudaMemcpyHostToDevice, s));
    SFCDD_CUDA_OK(cudaMemsetAsync(h->tmp, 0, (size_t)h->N * sizeof(double), s));
    SFCDD_CUDA_OK(cudaMemsetAsync(h->g0, 0, (size_t)h->nt0 * TILE * sizeof(double), s));
    TrsvArgs af = trsv_args(h, true, h->tmp, nullptr, LIST_MAIN);
    launch_trsv_fwd(af, h->st, s, wl.n - 1);
    SFCDD_CUDA_OK(cudaStreamSynchronize(s));
    // restore the substitution state: pending result slots, tickets at zero
    launch_fill_pending(h->ybuf, h->vtotal, s);
    launch_fill_pending(h->dbuf, h->vtotal, s);
    SFCDD_CUDA_OK(cudaMemsetAsync(wl.tf, 0, sizeof(unsigned long long), s));
    SFCDD_CUDA_OK(cudaMemsetAsync(wl.tb, 0, sizeof(unsigned long long), s));
    if (keep_l == 0) {
      ErrWord e{};
      SFCDD_CUDA_OK(cudaMemcpyAsync(&e, h->err, sizeof(ErrWord), cudaMemcpyDeviceToHost, s));
      SFCDD_CUDA_OK(cudaStreamSynchronize(s));
      SFCDD_CUDA_OK(cudaMemsetAsync(h->err, 0, sizeof(ErrWord), s));
      TRY(configure_substitution(h, 0, h->nsub_coarse));
      SFCDD_CUDA_OK(cudaMemcpyAsync(h->err, &e, sizeof(ErrWord), cudaMemcpyHostToDevice, s));
      SFCDD_CUDA_OK(cudaStreamSynchronize(s));
    }
  }
  ErrWord e{};
  SFCDD_CUDA_OK(cudaMemcpyAsync(&e, h->err, sizeof(ErrWord), cudaMemcpyDeviceToHost, s));
  SFCDD_CUDA_OK(cudaMemsetAsync(h->err, 0, sizeof(ErrWord), s));
  SFCDD_CUDA_OK(cudaStreamSynchronize(s));
  if (detail) *detail = e.index;
  return e.code;
}

int sfcdd_autotune(sfcdd_handle* h, int reps, sfcdd_tuning* out) {
  NvtxRange nvtx("sfcdd autotune");
  if (!h || reps < 1) return SFCDD_ERR_INVALID_ARG;
  cudaStream_t s = h->stream;
  const bool prof = h->profiling;
  long long saved[SFCDD_K_COUNT];
  memcpy(saved, h->launches, sizeof(saved));
  h->profiling = false;
  // the timed applies read a zero vector: the substitution streams the same
  // tiles whatever the values
  SFCDD_CUDA_OK(cudaMemsetAsync(h->tmp, 0, (size_t)h->N * sizeof(double), s));
  cudaEvent_t e0, e1;
  SFCDD_CUDA_OK(cudaEventCreate(&e0));
  SFCDD_CUDA_OK(cudaEventCreate(&e1));
  int best_l = h->nsub_local, best_c = h->nsub_coarse, cand = 0;
  float best = -1.f;
  int rc = SFCDD_OK;
  const int opts[4] = {1, 2, 4, 0};  // 0: whole-matrix local items
  for (int il = 0; il < 4 && rc == SFCDD_OK; ++il)
    for (int ic = 0; ic < 3 && rc == SFCDD_OK; ++ic) {
      const int sl = opts[il], sc = opts[ic];
      if (!valid_slabs(h->precision, sl, sc)) continue;
      if (sl == 0 && (!whole_fits(h->st, h->max_nt) || h->variant == SFCDD_COARSE_ONLY)) continue;
      rc = configure_substitution(h, sl, sc);
      if (rc != SFCDD_OK) break;
      Prof pf(h, s);
      for (int k = 0; k < 2; ++k) enqueue_apply(h, pf, h->tmp, h->z, nullptr);
      cudaEventRecord(e0, s);
      for (int k = 0; k < reps; ++k) enqueue_apply(h, pf, h->tmp, h->z, nullptr);
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
  memcpy(h->launches, saved, sizeof(saved));
  h->profiling = prof;
  if (rc != SFCDD_OK) return rc;
  int fi = 0;
  const int ec = check_err(h, &fi);
  if (ec != 0) return ec;
  TRY(configure_substitution(h, best_l, best_c));
  if (out) {
    out->slabs_local = best_l == 0 ? -1 : best_l;
    out->slabs_coarse = best_c;
    out->apply_ms = best / reps;
    out->candidates = cand;
  }
  return SFCDD_OK;
}

int sfcdd_apply_precond(sfcdd_handle* h, const double* g_dev, double* z_dev, int curve_order) {
  if (!h || !g_dev || !z_dev) return SFCDD_ERR_INVALID_ARG;
  cudaStream_t s = h->stream;
  Prof pf(h, s);
  if (curve_order) {
    enqueue_apply(h, pf, g_dev, z_dev, nullptr);
  } else {
    h->launches[SFCDD_K_VECTOR] += 2;
    launch_lex_to_curve(h->g, h->curve_code, g_dev, h->tmp, s);
    enqueue_apply(h, pf, h->tmp, h->tmp2, nullptr);
    launch_curve_to_lex(h->g, h->curve_code, h->tmp2, z_dev, s);
  }
  SFCDD_CUDA_OK(cudaGetLastError());
  pf.collect();
  int fi = 0;
  return check_err(h, &fi);
}

int sfcdd_get_info(const sfcdd_handle* h, sfcdd_info* info) {
  if (!h || !info) return SFCDD_ERR_INVALID_ARG;
  info->N = h->N;
  info->N0 = h->N0;
  info->d = h->d;
  info->P = h->P;
  info->q = h->q;
  info->nbits = h->nbits;
  info->tile = TILE;
  info->precision = h->precision;
  info->variant = h->variant;
  info->weighting = h->weighting;
  info->flexible = h->flexible;
  const long long esz = h->precision == SFCDD_FP64 ? 8 : (h->precision == SFCDD_FP32 ? 4 : 2);
  // both substitution copies (Lh and Lh^T / E_K)
  info->factor_bytes = h->variant == SFCDD_COARSE_ONLY ? 0 : 2 * h->ltile_elems * esz;
  info->coarse_bytes = h->variant == SFCDD_ONE_LEVEL ? 0 : 2 * h->ctile_elems * 8;
  info->setup_ms = h->setup_ms;
  return SFCDD_OK;
}

int sfcdd_get_curve(const sfcdd_handle* hc, unsigned long long* keys_dev, int* perm_dev) {
  sfcdd_handle* h = const_cast<sfcdd_handle*>(hc);
  if (!h) return SFCDD_ERR_INVALID_ARG;
  cudaStream_t s = h->stream;
  if (keys_dev) {
    unsigned* codes = nullptr;
    SFCDD_CUDA_OK(cudaMalloc(&codes, (size_t)h->N * sizeof(unsigned)));
    launch_keygen(h->g, keys_dev, codes, s);
    h->launches[SFCDD_K_KEYGEN] += 1;
    SFCDD_CUDA_OK(cudaStreamSynchronize(s));
    cudaFree(codes);
  }
  if (perm_dev) {
    launch_perm_lex(h->g, h->curve_code, perm_dev, s);
    h->launches[SFCDD_K_VECTOR] += 1;
  }
  SFCDD_CUDA_OK(cudaStreamSynchronize(s));
  return SFCDD_OK;
}

int sfcdd_get_partition(const sfcdd_handle* h, long long* start_host, long long* len_host,
                        double* omega_host) {
  if (!h) return SFCDD_ERR_INVALID_ARG;
  for (int i = 0; i < h->P; ++i) {
    if (start_host) start_host[i] = h->h_start[i];
    if (len_host) len_host[i] = h->h_len[i];
    if (omega_host) omega_host[i] = h->h_omega[i];
  }
  return SFCDD_OK;
}

int sfcdd_get_coarse_matrix(const sfcdd_handle* hc, double* A0_dev) {
  sfcdd_handle* h = const_cast<sfcdd_handle*>(hc);
  if (!h || !A0_dev) return SFCDD_ERR_INVALID_ARG;
  cudaStream_t s = h->stream;
  double* t = nullptr;
  SFCDD_CUDA_OK(cudaMalloc(&t, std::max<long long>(h->ctile_elems, 1) * sizeof(double)));
  const TileSetDev cts = coarse_view(h);
  launch_assemble_coarse(h->g, h->pd, h->curve_code, h->invpad, cts, h->stored[h->P], t, s);
  launch_unpack_dense(cts, 0, t, A0_dev, h->pd.crow, s);
  h->launches[SFCDD_K_COARSE_ASSEMBLE] += 1;
  h->launches[SFCDD_K_VECTOR] += 1;
  SFCDD_CUDA_OK(cudaStreamSynchronize(s));
  cudaFree(t);
  return SFCDD_OK;
}

int sfcdd_get_local_matrix(const sfcdd_handle* hc, int i, double* Ai_dev) {
  sfcdd_handle* h = const_cast<sfcdd_handle*>(hc);
  if (!h || !Ai_dev || i < 0 || i >= h->P) return SFCDD_ERR_INVALID_ARG;
  if (h->variant == SFCDD_COARSE_ONLY) return SFCDD_ERR_UNSUPPORTED;
  cudaStream_t s = h->stream;
  double* t = nullptr;
  SFCDD_CUDA_OK(cudaMalloc(&t, (size_t)h->stored[i] * TILE2 * sizeof(double)));
  const TileSetDev lts = local_view(h, i);
  PartDev pd = h->pd;
  pd.start = h->d_start + i;
  launch_assemble_local(h->g, pd, h->curve_code, h->invpad, lts, 0, 1, h->stored[i], t,
                        Store::F64, s);
  launch_unpack_dense(lts, 0, t, Ai_dev, nullptr, s);
  h->launches[SFCDD_K_ASSEMBLE] += 1;
  h->launches[SFCDD_K_VECTOR] += 1;
  SFCDD_CUDA_OK(cudaStreamSynchronize(s));
  cudaFree(t);
  return SFCDD_OK;
}

int sfcdd_set_profiling(sfcdd_handle* h, int enable) {
  if (!h) return SFCDD_ERR_INVALID_ARG;
  h->profiling = enable != 0;
  return SFCDD_OK;
}

int sfcdd_get_kernel_stats(sfcdd_handle* h, double* ms_total, long long* launches, int reset) {
  if (!h) return SFCDD_ERR_INVALID_ARG;
  for (int k = 0; k < SFCDD_K_COUNT; ++k) {
    if (ms_total) ms_total[k] = h->ms[k];
    if (launches) launches[k] = h->launches[k];
  }
  if (reset) {
    memset(h->ms, 0, sizeof(h->ms));
    memset(h->launches, 0, sizeof(h->launches));
  }
  return SFCDD_OK;
}

double sfcdd_kernel_work(const sfcdd_handle* h, int kc) {
  if (!h) return 0.0;
  const double esz = h->precision == SFCDD_FP64 ? 8 : (h->precision == SFCDD_FP32 ? 4 : 2);
  const bool loc = h->variant != SFCDD_COARSE_ONLY, crs = h->variant != SFCDD_ONE_LEVEL;
  // forward: the nonzero rows of the Lh tiles left of each row's diagonal
  // block; backward: the E tiles of the row's diagonal block and the nonzero
  // columns of the Lh^T tiles below it (coarse: whole tiles)
  const double t2 = (double)TILE2;
  const double lf = loc ? (double)h->fwd_elems_l * esz : 0.0;
  const double lb = loc ? (double)h->bwd_elems_l * esz : 0.0;
  const double cf = crs ? (double)h->fwd_tiles_c * t2 * 8.0 : 0.0;
  const double cbk = crs ? (double)h->bwd_tiles_c * t2 * 8.0 : 0.0;
  switch (kc) {
    case SFCDD_K_TRSV_FWD:
      return lf + cf;
    case SFCDD_K_TRSV_BWD:
      return lb + cbk;
    case SFCDD_K_STENCIL:
      return 16.0 * (double)h->N;
    case SFCDD_K_POTRF:
      return h->work_potrf;
    case SFCDD_K_TRSM:
      return h->work_trsm;
    case SFCDD_K_SYRK:
      return h->work_syrk;
    case SFCDD_K_COARSE_FACTOR:
      return h->work_coarse;
    default:
      return 0.0;
  }
}

int sfcdd_destroy(sfcdd_handle* h) {
  if (!h) return SFCDD_ERR_INVALID_ARG;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  destroy_impl(h);
  return SFCDD_OK;
}

const char* sfcdd_status_string(int st) {
  switch (st) {
    case SFCDD_OK: return "ok";
    case SFCDD_ERR_INVALID_ARG: return "invalid argument";
    case SFCDD_ERR_KEY_OVERFLOW: return "d * max(l) exceeds the 64 key bits";
    case SFCDD_ERR_NOMEM: return "out of device memory";
    case SFCDD_ERR_NOT_SPD: return "non-positive pivot in a Cholesky factorization";
    case SFCDD_ERR_MAXIT: return "maximum number of iterations reached";
    case SFCDD_ERR_NAN: return "NaN or Inf in the iteration";
    case SFCDD_ERR_TIMEOUT: return "bounded device wait timed out";
    case SFCDD_ERR_CUDA: return "CUDA runtime error";
    case SFCDD_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

}  // extern "C"
