// Curve order (Hilbert keys + radix sort) for callers that cannot allocate
// device memory: no cudaMalloc, no cudaFree, no allocating library call.
//
// Who needs it: code that runs while a CUDA stream is being captured into a
// graph (cudaMalloc is not allowed there), code inside a host that owns all
// device memory through its own pool, and latency-critical callers that must
// avoid cudaMalloc/cudaFree because they synchronise the device.  The sort's
// ping-pong buffers and digit histograms live in one file-scope device array
// of fixed size instead; the caller passes only the two outputs.
#include <cstdio>
#include <mutex>

#include "sfcdd_internal.cuh"

namespace sfcdd {
namespace {

constexpr int NOALLOC_MAX_POINTS = 1 << 18;  // 262,144 grid points
constexpr size_t round256(size_t v) { return (v + 255) / 256 * 256; }
// Layout: [sort keys: 8 B/pt][radix-sort temp][codes: 4 B/pt]
constexpr size_t KEYS_BYTES = round256((size_t)NOALLOC_MAX_POINTS * 8);
constexpr size_t TEMP_BYTES =
    round256((size_t)NOALLOC_MAX_POINTS * 12 + (size_t)256 * ((NOALLOC_MAX_POINTS + 4095) / 4096) * 4 + 256);
constexpr size_t CODES_BYTES = round256((size_t)NOALLOC_MAX_POINTS * 4);
constexpr size_t SCRATCH_BYTES = KEYS_BYTES + TEMP_BYTES + CODES_BYTES;  // about 6.4 MB

// Held by every GPU that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_scratch_addr[MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device with that device current (the host-side symbol is only a stand-in).
int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice", __FILE__, __LINE__);
  if (dev < 0 || dev >= MAX_DEVICES) return SFCDD_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return SFCDD_OK;
}

}  // namespace
}  // namespace sfcdd

using namespace sfcdd;

extern "C" int sfcdd_curve_order_noalloc(const int* levels, int d, unsigned long long* keys_dev,
                                         int* perm_dev, void* stream) {
  if (!levels || !keys_dev || !perm_dev || d < 1 || d > MAXD) return SFCDD_ERR_INVALID_ARG;
  // the bit counts first: with B <= 31 the point count below stays under 2^31
  int nbits = 0, B = 0;
  for (int j = 0; j < d; ++j) {
    if (levels[j] < 1 || levels[j] > 30) return SFCDD_ERR_INVALID_ARG;
    nbits = levels[j] > nbits ? levels[j] : nbits;
    B += levels[j];
  }
  if (d * nbits > 64) return SFCDD_ERR_KEY_OVERFLOW;
  if (B > 31) return SFCDD_ERR_UNSUPPORTED;
  long long N = 1;
  for (int j = 0; j < d; ++j) N *= (1ll << levels[j]) - 1;
  if (N > NOALLOC_MAX_POINTS) {
    fprintf(stderr,
            "sfcdd_curve_order_noalloc: %lld grid points exceed the static scratch limit of %d "
            "points; use sfcdd_setup_ex / sfcdd_get_curve instead\n",
            N, NOALLOC_MAX_POINTS);
    return SFCDD_ERR_INVALID_ARG;
  }
  GridDev g{};
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
  void* base = nullptr;
  const int rc = scratch_address(&base);
  if (rc != SFCDD_OK) return rc;
  unsigned char* sb = static_cast<unsigned char*>(base);
  unsigned long long* sort_keys = reinterpret_cast<unsigned long long*>(sb);
  void* temp = sb + KEYS_BYTES;
  unsigned* codes = reinterpret_cast<unsigned*>(sb + KEYS_BYTES + TEMP_BYTES);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // every scratch byte used below is written before it is read: nothing to clear
  launch_keygen(g, keys_dev, codes, s);
  SFCDD_CUDA_OK(cudaMemcpyAsync(sort_keys, keys_dev, (size_t)N * sizeof(unsigned long long),
                                cudaMemcpyDeviceToDevice, s));
  radix_sort_pairs(sort_keys, codes, (int)N, d * nbits, temp, s, nullptr);
  launch_perm_lex(g, codes, perm_dev, s);
  SFCDD_CUDA_OK(cudaGetLastError());
  return SFCDD_OK;
}
