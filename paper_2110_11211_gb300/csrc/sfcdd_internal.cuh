// Internal declarations of the sfcdd CUDA library (sm_103a).
//
// Data layout in HBM (all device memory is owned by the handle):
//  - curve_code[p]  (uint32, N): the point at curve position p, as its packed
//    lexicographic code  sum_j k_j << off_j  (off_j = sum_{j'>j} l_j').
//  - invpad[code]   (int32, 2^{sum l_j}): curve position of a code, -1 if the
//    code is not an interior grid point.
//  - PCG vectors (FP64, N) in curve order.
//  - local factors: per subdomain i the TILE x TILE tiles of its lower triangle
//    that lie inside the Cholesky envelope ("tile skyline"): tile row I keeps
//    tiles K = kmin[I]..I, where kmin[I] is the first tile column holding a
//    nonzero of A_i in any row of tile row I.  The factor's fill stays inside
//    each row's envelope, so every tile outside is an exact zero and is neither
//    stored nor touched.  Tile (I, K) sits at tbase[i] + (rowoff[I] + K - kmin[I])
//    TILE^2, row-major inside a tile.  After the setup the factor is kept in its
//    substitution form L = Lh blockdiag(L_KK): the first array holds
//    Lh_IK = L_IK L_KK^{-1} off the diagonal (its diagonal slot keeps L_KK^{-1},
//    which the solves do not read), a second array of the same layout holds
//    Lh_IK^T in slot (I, K) and E_K = L_KK^{-T} L_KK^{-1} in the diagonal slot.
//    Storage fp64, fp32 or bf16.  The coarse factor has the same layout in FP64
//    and is matrix index P; its rows follow a reverse Cuthill-McKee numbering of
//    the coarse blocks (PartDev::crow / cblock).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <vector>

#include "../../include/sfcdd.h"
#include <nvtx3/nvToolsExt.h>

namespace sfcdd {

constexpr int TILE = 64;          // tile edge of the packed factors
constexpr int TILE2 = TILE * TILE;
constexpr int MAXD = 8;

// Named range for profilers (NVTX; free when no tool is attached): setup
// stages, solves and tuning show up as spans on the host timeline.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Launches over many matrices: the matrix index runs over grid.y x grid.z
// (grid.y is limited to 65535); the excess CTAs of the last z slice return.
inline dim3 mat_grid(unsigned x, int nmat) {
  const unsigned n = nmat > 0 ? (unsigned)nmat : 1u;
  const unsigned y = n < 65535u ? n : 65535u;
  return dim3(x, y, (n + y - 1) / y);
}
#ifdef __CUDACC__
__device__ __forceinline__ int grid_mat() { return (int)(blockIdx.y + gridDim.y * blockIdx.z); }
#endif

// Grid description passed by value to kernels.
struct GridDev {
  int d;
  int N;
  int nbits;                 // curve resolution n = max_j l_j
  int lev[MAXD];
  int off[MAXD];             // bit offset of axis j inside a code
  int size[MAXD];            // 2^{l_j} - 1
  int stride[MAXD];          // lexicographic stride of axis j
  double w[MAXD];            // c_j * 4^{l_j}
  double diag;               // sum_j 2 w_j
};

// Partition description (eqs. sloc, enlarge, restr) passed by value.
struct PartDev {
  int N, P, q, g;            // g = floor(gamma)
  int f, r;                  // floor(N/P), N mod P
  const int* start;          // P: first curve position of Omega_i
  const int* len;            // P: N_i
  const double* omega;       // P: omega_i (or 1)
  // Numbering of the coarse unknowns in the coarse factor: coarse block b
  // (eq. restr order) is row crow[b], row r holds block cblock[r]; null: b = r.
  const int* crow;
  const int* cblock;
};

// Tilde subdomain of a curve position (eq. sloc, closed form).
__host__ __device__ inline int tilde_of(const PartDev& pd, int p) {
  const int big = pd.r * (pd.f + 1);
  return p < big ? p / (pd.f + 1) : pd.r + (p - big) / pd.f;
}
__host__ __device__ inline int tilde_off(const PartDev& pd, int t) {
  return t < pd.r ? t * (pd.f + 1) : pd.r * (pd.f + 1) + (t - pd.r) * pd.f;
}
__host__ __device__ inline int tilde_size(const PartDev& pd, int t) {
  return t < pd.r ? pd.f + 1 : pd.f;
}
// Coarse block index (eq. restr) of a curve position: tilde subdomain t cut
// into q blocks, the first (size mod q) one point longer.
__host__ __device__ inline int coarse_block_of(const PartDev& pd, int p) {
  const int t = tilde_of(pd, p);
  const int o = p - tilde_off(pd, t);
  const int n = tilde_size(pd, t);
  const int bf = n / pd.q, br = n % pd.q;
  const int big = br * (bf + 1);
  const int m = o < big ? o / (bf + 1) : br + (o - big) / bf;
  return t * pd.q + m;
}
// First curve position and size of coarse block b.
__host__ __device__ inline void coarse_block_range(const PartDev& pd, int b, int& start,
                                                   int& size) {
  const int t = b / pd.q, m = b % pd.q;
  const int n = tilde_size(pd, t);
  const int bf = n / pd.q, br = n % pd.q;
  start = tilde_off(pd, t) + (m < br ? m * (bf + 1) : br * (bf + 1) + (m - br) * bf);
  size = m < br ? bf + 1 : bf;
}
__device__ __forceinline__ int coarse_row(const PartDev& pd, int b) {
  return pd.crow ? __ldg(&pd.crow[b]) : b;
}
__device__ __forceinline__ int coarse_block_at(const PartDev& pd, int r) {
  return pd.cblock ? __ldg(&pd.cblock[r]) : r;
}

// Hilbert key (Sec. 3.2, Skilling's transform) of the point with lexicographic
// id `id`; also returns its packed code.  D = dimension.
template <int D>
__device__ __forceinline__ unsigned long long hilbert_key_of(const GridDev& g, int id,
                                                             unsigned& code) {
  unsigned long long X[D];
  code = 0;
  int rem = id;
#pragma unroll
  for (int j = D - 1; j >= 0; --j) {
    const int kj = rem % g.size[j] + 1;
    rem /= g.size[j];
    X[j] = (unsigned long long)kj << (g.nbits - g.lev[j]);
    code |= (unsigned)kj << g.off[j];
  }
  const int nb = g.nbits;
  if (nb > 0) {
    const unsigned long long top = 1ull << (nb - 1);
    for (unsigned long long Q = top; Q > 1; Q >>= 1) {  // undo excess work
      const unsigned long long low = Q - 1;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        if (X[i] & Q) {
          X[0] ^= low;  // invert
        } else {
          const unsigned long long t = (X[0] ^ X[i]) & low;  // exchange
          X[0] ^= t;
          X[i] ^= t;
        }
      }
    }
#pragma unroll
    for (int i = 1; i < D; ++i) X[i] ^= X[i - 1];  // Gray encode
    unsigned long long t = 0;
    for (unsigned long long Q = top; Q > 1; Q >>= 1)
      if (X[D - 1] & Q) t ^= Q - 1;
#pragma unroll
    for (int i = 0; i < D; ++i) X[i] ^= t;
  }
  unsigned long long key = 0;  // bits level by level, axis 0 first
  for (int b = nb - 1; b >= 0; --b) {
#pragma unroll
    for (int i = 0; i < D; ++i) key = (key << 1) | ((X[i] >> b) & 1ull);
  }
  return key;
}

// One subgrid problem of a batch: its grid, partition, and where its data
// sits in the batch-wide arrays (positions are local to the subgrid).
struct SubDesc {
  GridDev g;
  PartDev pd;      // start/len/omega point into the batch arrays at this subgrid
  int base;        // first batch-wide curve position / vector entry
  int ibase;       // offset of this subgrid's invpad table
  int g0base;      // offset of its coarse vector (nt0 * TILE doubles)
  int mat0;        // first local matrix; the coarse matrix is cmat
  int cmat;
  int N0;
};

// Tile-skyline set of several matrices.  Per-tile-row arrays are indexed by
// fb + I with fb = vbase[m] / TILE (the global tile-row index of row 0 of m).
struct TileSetDev {
  int nmat;
  const int* n;              // dimension of each matrix
  const int* nt;             // tiles per dimension
  const long long* tbase;    // element offset of the first tile
  const int* vbase;          // offset of the matrix's vector slices (nt*TILE doubles)
  const int* kmin;           // [fb + I] first stored tile column of tile row I
  const int* rowoff;         // [fb + I] tiles stored before tile row I in its matrix
  const int* colptr;         // [fb + K], [fb + K + 1]: range in colidx of rows I > K, kmin[I] <= K
  const int* colidx;         // those rows, ascending
  const int* lperm;          // [vbase + r] curve position of local row r (null: curve order)
  const int* linv;           // [vbase + o] local row of offset o in the range (null: curve order)
  // [fb + I] rows of tile row I's off-block tiles that may hold nonzeros: rows
  // nzr.. of every Lh tile left of the row's diagonal block are zero, and so are
  // columns nzr.. of their transposes (null: no such bound, read whole tiles)
  const int* nzr;
};

__device__ __forceinline__ long long tile_at(const TileSetDev& ts, long long tb, int fb, int I,
                                             int K) {
  return tb + ((long long)ts.rowoff[fb + I] + (K - ts.kmin[fb + I])) * (long long)(64 * 64);
}

// Device-side PCG scalars (one struct per handle).
struct PcgScalars {
  double bb;       // ||b||^2
  double rz;       // r^T z (current)
  double pq;       // p^T A p
  double alpha, beta;
  double rr;       // ||r||^2
  double rel;      // ||r|| / ||b||
  double rtol;
  double rz_old;   // r_{k+1}^T z_k (flexible beta)
  double true_rel; // ||b - A x|| / ||b|| recomputed at exit
  double grad[MAXD];
  int iter;
  int done;
  int status;
  int flexible;
  // optional record of the PCG coefficients (Lanczos estimate of the spectrum):
  // hist_alpha[k] = alpha_k, hist_beta[k] = beta_k for k < hist_cap
  double* hist_alpha;
  double* hist_beta;
  int hist_cap;
  // energy-norm stopping for the homogeneous problem (f = 0, solution 0):
  // ||x||_A^2 = -x^T r, converged when it falls below rtol^2 ||x_0||_A^2 = rtol^2 esq0
  int energy;
  double esq0;
};

// Reduction workspace: per-block partials + arrival counter.
struct ReduceWs {
  double* partial;           // nblocks * ncomp
  unsigned int* counter;
  int nblocks;
};

// Error word written by kernels: first failure wins.
struct ErrWord {
  int code;    // sfcdd_status
  int index;
};

// ---------------- host helpers (api.cu) ----------------
// Grid description from levels and coefficients (coeffs may be null = ones).
int make_grid(const int* levels, int d, const double* coeffs, GridDev& g, long long& N, int& B);
// eqs. sloc / enlarge / omegai on the host (gamma read as round(gamma 2^16)/2^16).
int partition_ranges(long long N, int P, double gamma, int weighting, std::vector<int>& start,
                     std::vector<int>& len, std::vector<double>& omega, int& gfloor);
// q of the "four levels coarser" rule, clamped to 1..floor(N/P).
int paper_q(long long N, int P);
// Substitution work lists over the matrices with include[m] != 0: rows ordered
// by relative progress (r + 1) / nt[m] (backward: from the last row), so every
// matrix advances at the same relative rate and each row follows its
// predecessors in its own matrix.
struct TrsvWork;
void build_worklists(const std::vector<int>& nt, const std::vector<char>& include,
                     const std::vector<int>& nsub, std::vector<TrsvWork>& wf,
                     std::vector<TrsvWork>& wb);
// Tile-skyline bookkeeping of nmat matrices from the envelope of every tile row
// (tfirst = first nonzero column of the tile row): per-row kmin/rowoff, stored
// tile counts, element offsets (local matrices in one buffer, coarse ones in
// another), column lists, per-step launch sizes and operation counts.
struct SkylineHost {
  std::vector<int> kmin, rowoff, colptr, colidx, stored, col_max_local, col_max_coarse;
  std::vector<long long> tbase;
  long long ltiles = 0, ctiles = 0;  // stored tiles in the local / coarse buffers
  int max_ltiles = 0, max_ctiles = 0;
  double potrf = 0, trsm = 0, syrk = 0, coarse = 0;
  // tiles read by one forward / backward substitution (local, coarse)
  long long fwd_tiles_l = 0, bwd_tiles_l = 0, fwd_tiles_c = 0, bwd_tiles_c = 0;
};
// cb[m] > 1: matrix m is solved with cb-tile diagonal blocks (its envelope is
// widened to whole blocks).
void build_skyline(const std::vector<int>& nt, const std::vector<int>& vbase,
                   const std::vector<char>& is_coarse, const std::vector<int>& cb,
                   const std::vector<int>& tfirst, SkylineHost& out);

// ---------------- kernels / launchers (defined in the .cu files) ----------------

// keys_sort.cu
void launch_keygen(const GridDev& g, unsigned long long* keys, unsigned* codes, cudaStream_t s);
size_t radix_sort_temp_bytes(int n);
void radix_sort_pairs(unsigned long long* keys, unsigned* vals, int n, int bits, void* temp,
                      cudaStream_t s, int* launches);
void launch_invpad_fill(const unsigned* curve_code, int* invpad, int n, cudaStream_t s);
void launch_perm_lex(const GridDev& g, const unsigned* curve_code, int* perm, cudaStream_t s);

// vector.cu
int vec_blocks(int n);
void launch_lex_to_curve(const GridDev& g, const unsigned* code, const double* in, double* out,
                         cudaStream_t s);
void launch_curve_to_lex(const GridDev& g, const unsigned* code, const double* in, double* out,
                         cudaStream_t s);
void launch_stencil(const GridDev& g, const unsigned* code, const int* invpad, const double* x,
                    double* y, int mode, PcgScalars* sc, ReduceWs ws, cudaStream_t s);
void launch_update_xr(int n, double* x, double* r, const double* p, const double* q,
                      PcgScalars* sc, ReduceWs ws, cudaStream_t s);
void launch_restrict(const PartDev& pd, const double* r, double* g0, const PcgScalars* sc,
                     cudaStream_t s);
// mode 0 additive, 1 one level, 2 coarse only.  With sc and dot: fused r^T z
// PCG finalize; with sc and !dot: only the early return after convergence.
void launch_prolong(const PartDev& pd, const TileSetDev& ts, int mode, const double* dvec,
                    const double* r, double* z, PcgScalars* sc, ReduceWs ws, cudaStream_t s,
                    bool dot = true);
// y = b - A x (sc: early return after convergence)
void launch_residual(const GridDev& g, const unsigned* code, const int* invpad, const double* b,
                     const double* x, double* y, PcgScalars* sc, ReduceWs ws, cudaStream_t s);
// z = t - v + w (eq. balSW from its parts), with sc: fused r^T z PCG finalize
void launch_combine_bal(int n, const double* t, const double* v, const double* w, const double* r,
                        double* z, PcgScalars* sc, ReduceWs ws, cudaStream_t s);
void launch_update_p(int n, const double* z, double* p, const PcgScalars* sc, cudaStream_t s);

// The vector phase of one PCG iteration in one cooperative launch (every CTA
// resident; two grid barriers): prolongation z = C^{-1} r with r^T z -> beta;
// p_new = z + beta p_old (double-buffered by iteration parity), q = A p_new and
// p^T q -> alpha; x += alpha p, r -= alpha q, ||r|| -> convergence; the coarse
// restriction g0 = R_0 r for the next iteration.  Each CTA owns the curve
// positions [range[c], range[c + 1]), whole coarse blocks when mode != 1.
struct FusedPcg {
  GridDev g;
  PartDev pd;
  TileSetDev ts;
  const unsigned* code;
  const int* invpad;
  const double* dvec;        // substitution results (local slices, coarse at vbase[P])
  double* x;
  double* r;
  double* z;
  double* p[2];              // p of even / odd iterations
  double* q;
  double* g0;
  PcgScalars* sc;
  double* part;              // [2 phases][nblocks][2] block partials
  ReduceWs ws;               // last-block reduction of the third phase
  unsigned* bar;             // grid barrier: arrivals since the solve started
  const int* range;          // [nblocks + 1]
  ErrWord* err;
  int mode;                  // 0 two-level, 1 one level, 2 coarse only
  int nblocks;
};
// CTAs one cooperative launch of the fused kernel can keep resident (0 on error).
int fused_pcg_blocks(int d);
int launch_fused_pcg(const FusedPcg& a, cudaStream_t s);
void launch_init_pcg(int n, const double* b, double* x, double* r, PcgScalars* sc, ReduceWs ws,
                     double rtol, int flexible, cudaStream_t s);
void launch_energy(int n, const double* x, const double* r, PcgScalars* sc, ReduceWs ws,
                   double rtol, int flexible, int init, cudaStream_t s);
void launch_true_residual(const GridDev& g, const unsigned* code, const int* invpad,
                          const double* b, const double* x, double* tmp, PcgScalars* sc,
                          ReduceWs ws, cudaStream_t s);
void launch_axpby(int n, double a, const double* x, double b, const double* y, double* out,
                  cudaStream_t s);
void launch_grad(const GridDev& g, const unsigned* code, const int* invpad, const double* lam,
                 const double* u, PcgScalars* sc, ReduceWs ws, cudaStream_t s);

// Launch accounting hook (implemented by the API layer): counts launches per
// kernel class and, when profiling, brackets them with CUDA events.
struct LaunchHook {
  virtual void before(int cls) = 0;
  virtual void after(int cls) = 0;
  virtual ~LaunchHook() {}
};

// factor.cu
enum class Store { F64 = 0, F32 = 1, BF16 = 2 };
// Envelopes: tfirst[fb + I] receives the smallest column index with a nonzero
// in any row of tile row I (initialised by launch_envelope_init).
void launch_envelope_init(const TileSetDev& ts, int nmat, int max_nt, int* tfirst, cudaStream_t s);
void launch_envelope_local(const GridDev& g, const PartDev& pd, const unsigned* code,
                           const int* invpad, const TileSetDev& ts, int nmat, int max_n, int* tfirst,
                           cudaStream_t s);
void launch_envelope_coarse(const GridDev& g, const PartDev& pd, const unsigned* code,
                            const int* invpad, int fb_coarse, int* tfirst, cudaStream_t s);
void launch_assemble_local(const GridDev& g, const PartDev& pd, const unsigned* code,
                           const int* invpad, const TileSetDev& ts, int mat0, int nmat, int max_tiles,
                           void* tiles, Store st, cudaStream_t s);
void launch_assemble_coarse(const GridDev& g, const PartDev& pd, const unsigned* code,
                            const int* invpad, const TileSetDev& cts, int ntiles, double* tiles,
                            cudaStream_t s);
// Blocked right-looking Cholesky of matrices [mat0, mat0+nmat) of the tile set,
// in place, over the stored tiles only; diagonal slots end up holding the
// inverse of the factor's diagonal block.  col_max[K] = largest number of rows
// I > K with kmin[I] <= K over the matrices (sizes the step-K launches).
// split = 4 (FP64 only) computes every panel and trailing tile product as four
// 16-row slabs on four CTAs (for few, long factorizations such as the coarse one).
// diag_cnt: one int per tile row of ts (indexed fb + I), zero on entry; the
// trailing update of step k factors diagonal tile k+1 once its last update is in.
void factor_tiles(const TileSetDev& ts, int mat0, int nmat, int max_nt, const int* col_max,
                  void* tiles, Store st, int* diag_cnt, ErrWord* err, cudaStream_t s,
                  LaunchHook* hook, int split = 1, bool tensor_cores = false,
                  bool bf16_operands = false);
// Substitution form of the factors of matrices [mat0, mat0+nmat) (after
// factor_tiles, same precision): every stored off-diagonal tile L_IK becomes
// Lh_IK = L_IK L_KK^{-1} in place, ut receives Lh_IK^T in the same slot and
// E_K = L_KK^{-T} L_KK^{-1} in the diagonal slot (ut has the layout of tiles).
// max_stored = largest stored tile count of one matrix (sizes the launch).
void unitize_tiles(const TileSetDev& ts, int mat0, int nmat, int max_stored, void* tiles, void* ut,
                   Store st, cudaStream_t s);
// The same with cb-tile diagonal blocks for a one-matrix FP64 tile set (the
// coarse factor, envelope widened to whole blocks): below-block tiles become
// Lh_IK = sum_k L_{I,k} X_{k,K} (X_J = inverse of the block-triangular
// diagonal block J) with Lh^T in ut; inside block J, ut(I, K) = E_J(I, K) and
// tiles(I, K) = E_J(K, I) for I > K, E_J = X_J^T X_J.  xs: scratch of
// ceil(nt / cb) cb^2 tiles; stored = stored tile count.
void unitize_blocks(const TileSetDev& ts, int nt, int cb, int stored, double* tiles, double* ut,
                    double* xs, cudaStream_t s);
void launch_convert_f32_bf16(const float* in, __nv_bfloat16* out, long long n, cudaStream_t s);
// Lexicographic numbering inside each local matrix: matrices [0, nmat) of ts,
// matrix m covers the cyclic range (mstart[m], ts.n[m]) of a problem with
// mN[m] points whose codes start at code + mcbase[m]; lbase[m] = sum of the
// earlier sizes.  keys/vals/temp: scratch of total entries (+ sort temp).
void local_order_lex(const TileSetDev& ts, int nmat, int max_n, const int* mstart, const int* mN,
                     const int* mcbase, const int* lbase, long long total, const unsigned* code,
                     unsigned long long* keys, unsigned* vals, void* temp, int* lperm, int* linv,
                     cudaStream_t s);
// rowmap (null: ts.linv of the matrix) maps an output row/column to its row in the tiles.
void launch_unpack_dense(const TileSetDev& ts, int m, const double* tiles, double* dense,
                         const int* rowmap, cudaStream_t s);
// Distinct coarse blocks adjacent to each coarse block (in eq. restr order):
// adj[b * maxdeg + k], k < deg[b]; deg[b] = -1 if more than maxdeg.
void launch_coarse_adjacency(const GridDev& g, const PartDev& pd, const unsigned* code,
                             const int* invpad, int maxdeg, int* adj, int* deg, cudaStream_t s);

// trsv.cu
struct TrsvWork {
  int mat;
  int row;   // tile row; -1: the whole matrix (one CTA sweeps all its rows)
  int slab;  // rows [64 / nsub * slab, 64 / nsub * (slab + 1)) of the tile row
};
// Where the right-hand side of a matrix comes from and which solve it belongs to:
// a local matrix reads rhs[rhs_base + (start + row) mod rhs_len] (a cyclic slice of
// its problem's curve-order vector), a coarse matrix reads g0[rhs_base + row].
struct MatDesc {
  int rhs_base;
  int rhs_len;
  int start;
  int coarse;   // 1: FP64 coarse factor tiles, 0: local factor tiles
  int sub;      // index of the PCG scalars (problem) the matrix belongs to
  int nsub;     // slabs per tile row in the substitutions (1, 2 local; 1, 4 coarse)
  int cb;       // tiles per unit diagonal block of the substitution form (1, or 4 coarse)
};
// Bit pattern (a signalling NaN) marking a substitution result slot as not yet
// written in the current launch.
constexpr unsigned long long TRSV_PENDING = 0x7FF4DEADBEEF0000ull;
void launch_fill_pending(double* p, long long n, cudaStream_t s);
// Whether whole-matrix substitution items fit local matrices of up to max_nt
// tile rows with factors stored as st: the matrix vector beside the launch's
// ring must stay within a CTA's shared memory (227 KB).
bool whole_fits(Store st, int max_nt);
struct TrsvArgs {
  TileSetDev ts;
  const MatDesc* md;           // per matrix
  const void* ltiles;          // local Lh tiles (unit diagonal blocks implied)
  const void* lut;             // local Lh^T tiles, diagonal slots hold E_K
  const double* ctiles;        // coarse Lh tiles, may be null if no coarse
  const double* cut;           // coarse Lh^T tiles with E_K on the diagonal
  const double* rhs;           // curve-order vector the local right-hand sides are sliced from
  const double* g0;            // coarse right-hand sides (coarse block order)
  const int* cblock;           // coarse block of each coarse factor row (null: identity)
  double* y;                   // forward results, per matrix vbase
  double* dout;                // backward results, per matrix vbase
  double* zc;                  // plain copy of the forward results (read by the backward)
  const TrsvWork* work;        // work list, dependency-safe order
  int nwork;
  unsigned long long* ticket;  // monotone ticket counter
  ErrWord* err;
  const PcgScalars* sc;        // per problem (md.sub); null: no early exit
  // > 0: the local matrices of the work list are whole-matrix items (row < 0),
  // each swept by one CTA through a shared-memory vector of this many doubles
  // (the largest local tile count times TILE); 0: row-slab items only
  int zv_doubles;
  // row-slab launches: 1 streams through a 64 KB ring (three CTAs per SM; the
  // single large problems), 0 through 32 KB (FP64 one tile, FP32 two, BF16 four:
  // more CTAs per SM for the many small matrices of a batch)
  int wide_ring;
};
// grid > 0 launches that many CTAs instead of one per work item (self-test only)
void launch_trsv_fwd(const TrsvArgs& a, Store st, cudaStream_t s, int grid = 0);
// Fills nzr[fb + I] of the local matrices [mat0, mat0 + nmat) (cb = 1) from the
// stored Lh tiles: one past the last row holding a nonzero bit pattern.
void launch_offblock_rows(const TileSetDev& ts, int mat0, int nmat, int max_nt, const void* tiles,
                          Store st, int* nzr, cudaStream_t s);
// FP64 transposed off-block tiles Lh_IK^T (slot (I, K) of ut, I > K, matrices
// [mat0, mat0 + nmat) with cb = 1) whose row bound nzr[I] is at most TILE / 2
// keep their nonzeros in the left half of every row: packs those halves into
// the first TILE * TILE / 2 elements of the slot (row stride TILE / 2), the
// layout the backward substitution streams them in.  After launch_offblock_rows.
void launch_pack_half_tiles(const TileSetDev& ts, int mat0, int nmat, int max_stored, double* ut,
                            const int* nzr, cudaStream_t s);
// Factorization and inversion of one 64 x 64 FP64 tile in place (self-test of the
// breakdown report: a non-positive pivot sets NOT_SPD with index m).
void launch_potrf_one(double* tile, ErrWord* err, int m, cudaStream_t s);
void launch_trsv_bwd(const TrsvArgs& a, Store st, cudaStream_t s);

}  // namespace sfcdd

#define SFCDD_CUDA_OK(expr)                                             \
  do {                                                                  \
    cudaError_t _e = (expr);                                            \
    if (_e != cudaSuccess) return ::sfcdd::cuda_fail(_e, #expr, __FILE__, __LINE__); \
  } while (0)

namespace sfcdd {
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);
}
